"""md_observables_noalloc: the observables reduction for callers that may
not allocate device memory (fixed device-memory pools, no cudaMalloc after
start-up).  Checked through the C ABI against the existing md_observables on
the same particles, twice in a row (the shared scratch must be reusable),
and against the oracle's observables (Sec. 2.3) of the same per-particle
arrays.  FP64 tolerance as in the other parity tests: 1e-11 relative per
array."""
import numpy as np
import pytest

from paper_2503_07526_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_07526_gb300 as pkg

    pkg.lib(build=True)
    return pkg


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_noalloc_observables_match_md_observables(pkg, oracle_mod):
    import torch

    s = synth.lj_system(10, seed=3)
    n = s["n"]
    g = pkg.System(pkg.make_params(n, s["L"], precision=pkg.MD_PREC_FP64), s["r"], s["v"])
    dev = dict(device="cuda", dtype=torch.float64)
    v, e, W = torch.empty((3, n), **dev), torch.empty(n, **dev), torch.empty((6, n), **dev)
    mass = torch.ones(n, **dev)
    out = torch.full((12,), float("nan"), **dev)
    for steps in (3, 7):  # two calls in a row, different states
        g.step(steps)
        g.particles_device(v=v, epot=e, W=W)
        pkg.observables_noalloc(s["L"] ** 3, v, e, W, mass, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = g.observables()
        assert got[0] == pytest.approx(want["U"], rel=1e-11)
        assert got[1] == pytest.approx(want["K"], rel=1e-11)
        assert got[2] == pytest.approx(want["T"], rel=1e-11)
        assert rel(got[3:9], want["sigma"]) <= 1e-11
        assert rel(got[9:12], want["q"]) <= 1e-11
        ora = oracle_mod.observables(s["L"] ** 3, np.ones(n), v.cpu().numpy(), e.cpu().numpy(), W.cpu().numpy())
        assert got[0] == pytest.approx(ora[0], rel=1e-11)
        assert got[1] == pytest.approx(ora[1], rel=1e-11)
        assert rel(got[3:9], ora[3:9]) <= 1e-11
        assert rel(got[9:12], ora[9:12]) <= 1e-11
        out.fill_(float("nan"))


def test_noalloc_rejects_oversized_input(pkg):
    import torch

    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.MdError):  # n beyond the entry point's 2^27 - 1 maximum
        pkg._lib._check(pkg.lib().md_observables_noalloc(1 << 27, 1.0, t.data_ptr(), t.data_ptr(), t.data_ptr(),
                                                          t.data_ptr(), t.data_ptr(), 0))
