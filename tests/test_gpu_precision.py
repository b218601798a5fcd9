"""Error of each population storage type over the full tgv2d workload (D2Q9
2048^2, thermal Taylor-Green vortex with a Gaussian density/temperature pulse,
tau = 0.6, T0 = 0.1, 10,000 steps) against the FP64 path, which itself
matches the FP64 oracle to 1e-12 per step (test_gpu_parity.py).  Needs a
GB300.

Bounds (max |d| / max |ref| for rho and T, |d u| in units of c, relative
mass drift), about twice the errors measured once for each storage type:

  storage  step 1000: rho / u / T       step 10000: rho / u / T   mass drift
  FP32     3e-5 / 3e-6 / 5e-5           2e-4 / 1e-4 / 5e-4        1e-6
  FP16     6e-3 / 5e-3 / 6e-3           3e-2 / 2e-2 / 3e-2        3e-3
  BF16     5e-2 / 4e-2 / 6e-2           1.5e-1 / 1e-1 / 2e-1      1.2e-2
"""
import numpy as np
import pytest

from paper_2501_00620_gb300 import workloads as W

try:
    from paper_2501_00620_gb300 import lbm
except ImportError as _e:
    lbm = None
    _IMPORT_ERROR = _e

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _library_loaded():
    if lbm is None:
        raise _IMPORT_ERROR


BOUNDS = {  # storage: {step: (rho, u, T)}, mass drift at the last step
    "f32": ({1000: (3e-5, 3e-6, 5e-5), 10000: (2e-4, 1e-4, 5e-4)}, 1e-6),
    "f16": ({1000: (6e-3, 5e-3, 6e-3), 10000: (3e-2, 2e-2, 3e-2)}, 3e-3),
    "bf16": ({1000: (5e-2, 4e-2, 6e-2), 10000: (1.5e-1, 1e-1, 2e-1)}, 1.2e-2),
}


def run(dtype, checkpoints):
    c = W.CONFIGS["tgv2d"]
    rho, u, T = W.fields_for("tgv2d")
    g = lbm.Simulation(2, c["nx"], c["ny"], 1, tau=c["tau"], T0=c["T0"], bc=c["bc"], dtype=dtype,
                       thermal=c["thermal"])
    g.init(rho, u, T)
    m0 = g.diagnostics()[0]
    out, done = {}, 0
    for k in checkpoints:
        g.step(k - done)
        done = k
        out[k] = g.moments()
    drift = abs(g.diagnostics()[0] / m0 - 1)
    g.close()
    return out, drift


def test_storage_error_over_the_full_tgv2d_run():
    steps = (1000, 10000)
    ref, _ = run("f64", steps)
    for dtype, (bounds, drift_max) in BOUNDS.items():
        got, drift = run(dtype, steps)
        for k in steps:
            (rr, ur, Tr), (rg, ug, Tg) = ref[k], got[k]
            e_rho = np.abs(rg - rr).max() / np.abs(rr).max()
            e_u = np.abs(ug - ur).max()
            e_T = np.abs(Tg - Tr).max() / np.abs(Tr).max()
            b = bounds[k]
            assert e_rho < b[0] and e_u < b[1] and e_T < b[2], (dtype, k, e_rho, e_u, e_T)
        assert drift < drift_max, (dtype, drift)
