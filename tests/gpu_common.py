"""Shared helpers of the GPU parity tests: running the oracle beside the CUDA path
on the same seeded inputs, and the oracle's local (patch) evaluation used to check
sampled nodes of full-size workloads."""

import numpy as np
import pytest

from oracle import lattices as OL
from oracle import lbm as O
from paper_1712_08288_gb300 import binding as B


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # the library must load: a missing build is an error, not a skip
    B.lib()
    return torch


def oracle_sim(w, scheme=(0.0, 1.0, 0.0, 1.0), links=None):
    lat = OL.BY_NAME[w["lattice"]]
    return O.Simulation(lat, w["shape"], w["S"], w.get("rho0", 1.0), w["solid"],
                        links if links is not None else w["links"], scheme=scheme,
                        force=w.get("force", (0.0, 0.0, 0.0)), skew=w.get("skew", (0, 0)))


def gpu_sim(w, precision="f64", scheme=(0.0, 1.0, 0.0, 1.0), links=None, allow_nonconvex=True):
    ww = dict(w)
    if links is not None:
        ww["links"] = links
    return B.from_workload(ww, precision, scheme, allow_nonconvex=allow_nonconvex)


def rel_err(a, b, mask=None):
    """||a - b||_2 / ||b||_2 over the masked entries."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if mask is not None:
        a, b = a[..., mask], b[..., mask]
    return float(np.sqrt(((a - b) ** 2).sum()) / np.sqrt((b ** 2).sum()))


def entry_err(a, b, mask=None):
    """max_k |a_k - b_k| / max_k |b_k| over the masked entries: the bound on every
    single entry, relative to the largest entry of the reference."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if mask is not None:
        a, b = a[..., mask], b[..., mask]
    return float(np.abs(a - b).max() / np.abs(b).max())


def check_close(a, b, tol, mask=None, label=""):
    """Element-wise parity: every compared entry satisfies |a_k - b_k| <= tol max|b|
    (the per-entry bound), and the whole set ||a - b||_2 <= tol ||b||_2.  Non-finite
    entries fail.  Prints both figures and the worst entry; returns (entry, norm)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if mask is not None:
        a, b = a[..., mask], b[..., mask]
    assert a.shape == b.shape, (a.shape, b.shape)
    assert np.isfinite(a).all(), "%s: non-finite entries" % label
    d = np.abs(a - b)
    scale = np.abs(b).max()
    entry = float(d.max() / scale)
    norm = float(np.sqrt((d ** 2).sum()) / np.sqrt((b ** 2).sum()))
    worst = np.unravel_index(int(np.argmax(d)), d.shape)
    print("parity %s: per-entry %.3e, norm %.3e (tol %.1e; worst entry %s: %.17g vs %.17g)"
          % (label, entry, norm, tol, tuple(int(v) for v in worst), a[worst], b[worst]))
    assert entry <= tol, "%s: per-entry error %.3e > %.1e at %s" % (label, entry, tol, worst)
    assert norm <= tol, "%s: norm error %.3e > %.1e" % (label, norm, tol)
    return entry, norm


def check_fd(fd, g, rtol, floor, label=""):
    """A gradient entry against its central difference: |fd - g| <= rtol |fd| + floor,
    floor the difference quotient's own rounding (stated by the caller)."""
    err = abs(fd - g)
    print("fd %s: fd %.10e adjoint %.10e rel %.3e (floor %.1e)"
          % (label, fd, g, err / abs(fd) if fd else float("inf"), floor))
    assert err <= rtol * abs(fd) + floor, (label, fd, g)


def deviation(f, lat):
    """Population deviations g = f - w rho0 (rho0 = 1)."""
    return f - lat.w[:, None]


def patch_reference(w, f0_fn, centres, k, scheme):
    """f(x_c, t = k) at each centre, computed by the oracle on a local patch.

    The patch holds the nodes within distance R = k + 2 of the centre (periodic
    images, skew included) with its outer layer made solid; cut links of the real
    geometry keep their wall fraction and velocity, artificial links toward the
    outer layer get q = 1/2.  After k steps the corruption from the artificial
    layer has moved at most k nodes inward, so the centre is exact.
    f0_fn(idx) returns the initial full populations (Q, len(idx)) of global nodes.
    """
    lat = OL.BY_NAME[w["lattice"]]
    shape = w["shape"]
    skew = tuple(w.get("skew", (0, 0)))
    nx, ny, nz = shape
    R = k + 2
    three_d = lat.D == 3
    Pz = 2 * R + 1 if three_d else 1
    P = 2 * R + 1
    lk = w["links"]
    link_map = {}
    for idx, (n, d) in enumerate(zip(lk["node"].tolist(), lk["d"].tolist())):
        link_map[(n, d)] = idx
    out = []
    for c in centres:
        cx, cy, cz = c % nx, (c // nx) % ny, c // (nx * ny)
        oz, oy, ox = np.meshgrid(np.arange(Pz) - (R if three_d else 0), np.arange(P) - R,
                                 np.arange(P) - R, indexing="ij")
        gidx = O.wrapped_index(shape, skew, cx + ox.ravel(), cy + oy.ravel(), cz + oz.ravel())
        solid = np.asarray(w["solid"], bool)[gidx].copy()
        px, py, pz = ox.ravel() + R, oy.ravel() + R, oz.ravel() + (R if three_d else 0)
        edge = (px == 0) | (px == P - 1) | (py == 0) | (py == P - 1)
        if three_d:
            edge |= (pz == 0) | (pz == Pz - 1)
        solid |= edge
        pshape = (P, P, Pz)
        nbr = O.neighbour_table(lat, pshape, (0, 0))
        node, dd, qq, uw = [], [], [], []
        for d in range(1, lat.Q):
            for pn in np.nonzero(~solid & solid[nbr[d]])[0]:
                key = (int(gidx[pn]), d)
                node.append(pn)
                dd.append(d)
                if key in link_map:
                    j = link_map[key]
                    qq.append(lk["q"][j])
                    uw.append(np.asarray(lk["uw"][j], float))
                else:
                    qq.append(0.5)
                    uw.append(np.zeros(3))
        links = dict(node=np.array(node, np.int64), d=np.array(dd, np.int64),
                     q=np.array(qq, float), uw=np.array(uw, float).reshape(-1, 3))
        sim = O.Simulation(lat, pshape, w["S"], w.get("rho0", 1.0), solid, links, scheme=scheme,
                           force=w.get("force", (0.0, 0.0, 0.0)))
        f = f0_fn(gidx)
        f[:, solid] = np.nan
        sim.f = f
        sim.step(k)
        centre_local = R + P * (R + P * (R if three_d else 0))
        out.append(sim.f[:, centre_local].copy())
    return np.array(out).T    # (Q, len(centres))
