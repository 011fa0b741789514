"""Time step and SSP-RK3 stage (test infrastructure: oracle).

* dt = CFL * min_q dx_q / (2^(d-1) (2M - 1) lambda_q), lambda_q the largest
  |v_a| + c over the element's mean values (eqs. cfl-condition,
  euler-max-eigenvalue); dx_q is the smallest element edge.
* SSP-RK3 in Shu-Osher form, stage uout = a u0 + b (us + dt R(us)) with
  (a, b) = (0, 1), (3/4, 1/4), (1/3, 2/3). (The paper integrates with SSP-RK(5,4);
  the third-order scheme is used for the workloads here.)
"""
import numpy as np

from .blended import blended_rhs
from .euler import max_wave_speed

RK3_STAGES = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))


def cfl_dt(U, cfg):
    lam = max_wave_speed(U, cfg.gamma).max()
    return cfg.cfl * min(cfg.dx) / (2 ** (cfg.dim - 1) * (2 * cfg.M - 1) * lam)


def rk_stage(U0, Us, a, b, dt, cfg, frozen=None):
    return a * U0 + b * (Us + dt * blended_rhs(Us, cfg, frozen=frozen))


def rk3_step(U, cfg, dt=None):
    if dt is None:
        dt = cfl_dt(U, cfg)
    Us = U
    for a, b in RK3_STAGES:
        Us = rk_stage(U, Us, a, b, dt, cfg)
    return Us, dt
