"""Shared test helpers: map the CUDA path's float32 configuration onto the
oracle's (the oracle consumes exactly the same float32 input values)."""
import numpy as np

import oracle as O

FLOAT_FIELDS = ["kappa", "beta", "conf_c", "warp_lambda", "t_near", "t_far", "eps", "bias_alpha", "m_min", "r_mult"]


def f32(x):
    return float(np.float32(x))


def oracle_config(rc=None, **over):
    """OracleConfig with the float32-rounded values of a RasterConfig."""
    from paper_2512_11800_gb300 import RasterConfig
    rc = rc or RasterConfig()
    kw = {k: f32(getattr(rc, k)) for k in FLOAT_FIELDS}
    kw.update(n=rc.n, n_intervals=rc.n_intervals, bg=tuple(f32(b) for b in rc.bg))
    kw.update(over)
    return O.OracleConfig(**kw)
