"""GB300 (sm_103a) PIC-MCC electron hot path of Wang, Sun & Teunissen,
arXiv 2110.14494: velocity-Verlet push, null-collision Monte Carlo,
fixed-point CIC deposit, super-particle merge/split, multigrid Poisson and
Monte Carlo swarms, behind the C ABI of include/picmcc.h, and a BF16
surrogate of the swarms' transport data."""
from . import picmcc  # noqa: F401
from .picmcc import (PicContext, PicError, mlp_features, mlp_fold_standardization, mlp_forward,  # noqa: F401
                     mlp_loss_grad, mlp_train, poisson_axi_solve, poisson_solve, swarm_autotune, swarm_run)
