"""Time step and SSP-RK3 stage (test infrastructure: oracle).

* dt = CFL * min_q dx_q / (2^(d-1) (2M - 1) lambda_q), lambda_q the largest
  |v_a| + c over the element's mean values (eqs. cfl-condition,
  euler-max-eigenvalue); dx_q is the smallest element edge.
* SSP-RK3 in Shu-Osher form, stage uout = a u0 + b (us + dt R(us)) with
  (a, b) = (0, 1), (3/4, 1/4), (1/3, 2/3), used for the workloads here.
* SSP-RK(5,4), the integrator of the paper's runs (Sec. 3): five stages, fourth
  order, in the Shu-Osher form of Spiteri & Ruuth (2002),
  u_i = sum_k alpha_ik u_k + beta_ik dt L(u_k), k < i, u_0 = u^n, u^(n+1) = u_5.
"""
import numpy as np

from .blended import blended_rhs
from .euler import max_wave_speed

RK3_STAGES = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))

# Spiteri & Ruuth (2002), SSP-RK(5,4): rows i = 1..5, columns k = 0..i-1
SSPRK54_ALPHA = (
    (1.0,),
    (0.444370493651235, 0.555629506348765),
    (0.620101851488403, 0.0, 0.379898148511597),
    (0.178079954393132, 0.0, 0.0, 0.821920045606868),
    (0.0, 0.0, 0.517231671970585, 0.096059710526147, 0.386708617503269),
)
SSPRK54_BETA = (
    (0.391752226571890,),
    (0.0, 0.368410593050371),
    (0.0, 0.0, 0.251891774271694),
    (0.0, 0.0, 0.0, 0.544974750228521),
    (0.0, 0.0, 0.0, 0.063692468666290, 0.226007483236906),
)


def shu_osher_step(u, L, dt, alpha, beta):
    """One step of an explicit RK method in Shu-Osher form: stages
    u_i = sum_k alpha[i-1][k] u_k + beta[i-1][k] dt L(u_k); returns the last stage.
    L is evaluated once per stage value that some beta uses."""
    us, Ls = [u], {}
    for i in range(1, len(alpha) + 1):
        acc = 0.0
        for k in range(i):
            a, b = alpha[i - 1][k], beta[i - 1][k]
            if a != 0.0:
                acc = acc + a * us[k]
            if b != 0.0:
                if k not in Ls:
                    Ls[k] = L(us[k])
                acc = acc + b * dt * Ls[k]
        us.append(acc)
    return us[-1]


def ssprk54_step(U, cfg, dt=None):
    if dt is None:
        dt = cfl_dt(U, cfg)
    return shu_osher_step(U, lambda X: blended_rhs(X, cfg), dt, SSPRK54_ALPHA, SSPRK54_BETA), dt


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
