// Single-precision electron push (FMA contraction allowed).
#include "push_impl.cuh"
template struct pic::PushLaunch<float>;
template struct pic::BatchLaunch<float>;
