"""Helpers shared by the GPU parity tests: norm-wise errors and sampled-window
checks of large lattices against the oracle."""
import numpy as np

import oracle


def normwise(got, ref):
    """max |got - ref| / max |ref| (per field), robust to near-zero fields."""
    scale = np.abs(ref).max()
    if scale == 0:
        return np.abs(got - ref).max()
    return np.abs(got - ref).max() / scale


def window_indices(shape, center, half):
    """Periodic index arrays of a window of edge 2*half+1 around center."""
    idx = []
    for n, c in zip(shape, center):
        if n == 1:
            idx.append(np.array([0]))
        else:
            idx.append((np.arange(c - half, c + half + 1)) % n)
    return idx


def take_window(a, idx):
    """a: (k, nz, ny, nx) -> window (k, wz, wy, wx)."""
    iz, iy, ix = idx
    return a[:, iz][:, :, iy][:, :, :, ix]


def check_windows(d, f0, b0, f1, b1, tau, T0, thermal, n_windows=6, half=5, seed=0, model="bump"):
    """f0/b0: emitted state at t (full lattice, FP64 planes); f1/b1: the GPU's
    emitted state at t+1.  For random windows, restart the oracle from the
    window of (f0, b0), take one step and compare the window interior (sites
    at distance >= 2 from the window edge, where the periodic window is
    exact) with f1/b1.  Returns the worst norm-wise errors (f, b)."""
    rng = np.random.default_rng(seed)
    shape = f0.shape[1:]
    worst_f = worst_b = 0.0
    for _ in range(n_windows):
        center = [int(rng.integers(0, n)) for n in shape]
        idx = window_indices(shape, center, half)
        wf, wb = take_window(f0, idx), take_window(b0, idx)
        wz, wy, wx = wf.shape[1:]
        s = oracle.Sim(d, wx, wy, wz, tau=tau, T0=T0, thermal=thermal, model=model)
        s.set_emitted(wf, wb)
        s.step(1)
        of, ob = s.emitted()
        inner = tuple(slice(2, n - 2) if n > 1 else slice(0, 1) for n in (wz, wy, wx))
        gf, gb = take_window(f1, idx), take_window(b1, idx)
        sl = (slice(None),) + inner
        worst_f = max(worst_f, normwise(gf[sl], of[sl]))
        worst_b = max(worst_b, np.abs(gb[sl] - ob[sl]).max() / max(np.abs(ob[sl]).max(), 1e-3))
    return worst_f, worst_b
