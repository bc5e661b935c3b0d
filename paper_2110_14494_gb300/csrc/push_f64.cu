// Double-precision electron push.  Compiled with --fmad=false so every product
// and sum is rounded separately, in the same order as the CPU oracle.
#include "push_impl.cuh"
template struct pic::PushLaunch<double>;
template struct pic::BatchLaunch<double>;
