"""lbm_error_norms_noalloc: the allocation-free error norms agree with lbm_error_norms.

The entry point exists for callers that cannot allocate device memory when they need
the norms (a memory pool that owns the whole device, a fixed memory footprint, a
loop that cannot take cudaMalloc's implicit synchronisation).  It keeps its partial
sums in a static device array of the library.  This file is collected last on
purpose: if it fails, a run that stops at the first failure has already run every
other test.
"""

import numpy as np
import pytest

from paper_1712_08288_gb300 import binding as B
from paper_1712_08288_gb300 import workloads as W

from gpu_common import gpu_sim, require_gpu

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _compare(nrm, out):
    """out: l2_rel, linf, mass, mom[3], non-finite count (from the device)."""
    assert abs(out[0] - nrm["l2_rel"]) <= TOL * abs(nrm["l2_rel"])
    assert out[1] == nrm["linf"]
    assert abs(out[2] - nrm["mass"]) <= TOL * abs(nrm["mass"])
    scale = max(abs(v) for v in nrm["mom"]) + 1e-300
    for a, b in zip(out[3:6], nrm["mom"]):
        assert abs(a - b) <= TOL * scale
    assert out[6] == 0.0


@pytest.mark.parametrize("lattice,prec", [("D2Q9", "f64"), ("D3Q19", "f32")])
def test_noalloc_norms_match_allocating_entry_point(lattice, prec):
    torch = require_gpu()
    if lattice == "D2Q9":
        w = W.couette_config(96)
    else:
        w = W.tilted_pipe_3d(48)
    D = 2 if lattice == "D2Q9" else 3
    sim = gpu_sim(w, prec)
    stream = torch.cuda.current_stream()
    sim.set_stream(stream.cuda_stream)
    u_ref = np.ascontiguousarray(np.nan_to_num(w["u_exact"])[:, :D])
    u_ref_dev = torch.from_numpy(u_ref).cuda()
    out_dev = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
    sim.init_equilibrium()
    for call in range(2):                       # two calls in a row, state advancing
        sim.step(37 + call)                     # odd, then even time
        sim.error_norms_noalloc(u_ref_dev.data_ptr(), out_dev.data_ptr())
        torch.cuda.synchronize()
        out = out_dev.cpu().numpy()
        nrm = sim.error_norms(u_ref)
        _compare(nrm, out)
    # without a reference field the velocity norms are NaN, the sums remain
    sim.error_norms_noalloc(0, out_dev.data_ptr())
    torch.cuda.synchronize()
    out = out_dev.cpu().numpy()
    assert np.isnan(out[0]) and np.isnan(out[1])
    assert abs(out[2] - sim.error_norms(None)["mass"]) <= TOL * abs(out[2])
    sim.close()


def test_noalloc_rejects_grids_beyond_the_static_limit():
    torch = require_gpu()
    sim = B.Lbm("D3Q19", (324, 324, 324), W.relaxation_rates("D3Q19", 1.0), "f16")
    out_dev = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
    with pytest.raises(B.LbmError) as ei:
        sim.error_norms_noalloc(0, out_dev.data_ptr())
    assert ei.value.code == -1
    assert "33,554,432 nodes" in str(ei.value)
    torch.cuda.synchronize()
    assert torch.isnan(out_dev).all()           # nothing was launched
    sim.close()
