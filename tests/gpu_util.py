"""Helpers shared by the GPU parity tests: seeded problems, oracle calls and
the relative-L2 metric."""
import numpy as np
import torch

import oracle as orc
from paper_2505_14372_b300 import Context, Geometry


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def problem(seed, S, K, N, H, W, B, loss="amplitude", eps=1e-3, c=0.0, bandlimit=2 / 3, dz=10.0,
            edge=False):
    """Seeded synthetic problem: a smooth-ish probe, a weak phase object with
    some absorption, random positions (optionally touching the object edges)."""
    rng = np.random.default_rng(seed)
    y = np.arange(N) - N / 2
    r2 = (y[:, None] ** 2 + y[None, :] ** 2) / (N / 6) ** 2
    base = np.exp(-r2) * np.exp(1j * 0.5 * r2)
    P = np.stack([base * (1 + 0.3 * rng.standard_normal((N, N))) * np.exp(1j * 0.3 * rng.standard_normal((N, N)))
                  for _ in range(K)]) * 3.0
    O = np.exp(1j * 0.4 * rng.standard_normal((S, H, W))) * (0.9 + 0.1 * rng.random((S, H, W)))
    pos = np.stack([rng.uniform(-0.49, H - N - 0.51, B), rng.uniform(-0.49, W - N - 0.51, B)], 1)
    if edge and B >= 4:
        pos[0] = [0.0, 0.0]
        pos[1] = [H - N, W - N]
        pos[2] = [-0.5, 0.25]          # rounds up to 0
        pos[3] = [H - N + 0.4999, 3.5]  # rounds down to H - N; 3.5 rounds to 4
    pos = pos.astype(np.float32)
    geom = Geometry(S=S, K=K, N=N, H=H, W=W, dx=0.1, lam=0.0197, dz=tuple([dz] * (S - 1)),
                    bandlimit=bandlimit, loss=loss, eps=eps, c=c)
    og = orc.Geom(S=S, K=K, h=N, w=N, H=H, W=W, dx=0.1, lam=0.0197, dz=geom.dz, bandlimit=bandlimit,
                  loss={"amplitude": 0, "anscombe": 0, "poisson": 1}[loss], eps=eps, c=c)
    return geom, og, P.astype(np.complex64), O.astype(np.complex64), pos


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy()
