"""GPU test of the pipelined host-to-host step: fields in pinned host memory,
copied in, run through the five operators and copied back on three streams,
give the same results (bitwise) as the operators applied on one stream, over
several back-to-back steps whose inputs change between steps."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.mark.parametrize("N,nlev,ld", [(32, 5, 8), (80, 137, 140)])
def test_hoststep_matches_device_operators(torch, pfvm, N, nlev, ld):
    from paper_1908_07038_gb300.hoststep import HostStep
    fvm = pfvm(N)
    V = fvm.nnodes
    gen = torch.Generator().manual_seed(5)
    steps = 3
    hin = [{n: torch.randn((V, ld), generator=gen).pin_memory() for n in ("f", "u", "v")} for _ in range(steps)]
    hs = HostStep(fvm, nlev, ld, torch.float32)
    assert hs.h2d_bytes == 3 * V * ld * 4 and hs.d2h_bytes == 7 * V * ld * 4
    hout = [{n: torch.full((V, ld), 7.0).pin_memory() for n in hs.outputs} for _ in range(steps)]
    hs.begin()
    for s in range(steps):
        hs.enqueue(hin[s], hout[s])
    hs.synchronize()
    for s in range(steps):
        f, u, v = (hin[s][n].cuda() for n in ("f", "u", "v"))
        want = {}
        want["gx"], want["gy"] = fvm.gradient(f, nlev)
        want["lap"] = fvm.laplacian(f, nlev)
        want["du"], want["dv"] = fvm.divergence_adjoint(f, nlev)
        want["div"] = fvm.divergence(u, v, nlev)
        want["ga"] = fvm.gradient_adjoint(u, v, nlev)
        torch.cuda.synchronize()
        for n in hs.outputs:
            got = hout[s][n][:, :nlev]
            assert torch.equal(got, want[n][:, :nlev].cpu()), (s, n)


def test_hoststep_rejects_bad_host_buffers(torch, pfvm):
    from paper_1908_07038_gb300.hoststep import HostStep
    fvm = pfvm(16)
    hs = HostStep(fvm, 4, 4, torch.float32, ops=("gradient",))
    assert hs.inputs == ("f",) and hs.outputs == ("gx", "gy")
    good = torch.zeros((fvm.nnodes, 4)).pin_memory()
    with pytest.raises(ValueError):
        hs.enqueue({"f": torch.zeros((fvm.nnodes, 5))}, {"gx": good, "gy": good.clone()})
    with pytest.raises(ValueError):
        hs.enqueue({"f": good.double()}, {"gx": good, "gy": good.clone()})
    with pytest.raises(ValueError):
        HostStep(fvm, 4, 4, torch.float32, ops=("curl",))
