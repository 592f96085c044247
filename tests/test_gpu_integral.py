"""GPU: the FP64 volume-weighted sums (``atlas_fvm_integral``) against the
oracle's correctly rounded sums, within the error bound of the kernel's
summation (four interleaved accumulators over each block's chunk of nodes,
the first also taking the last < 8 nodes, then the block partials in order:
(chunk/4 + 10 + blocks) eps sum|V x|);
conservation of the FP64 divergence and curl on the sphere; node ranges
and partitions; empty ranges; BF16 storage."""
import numpy as np
import pytest

import synthetic
from oracle import oracle

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _bound(torch, V, x, count):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    maxb = 8 * sms
    chunk = -(-count // maxb) if count else 0
    blocks = -(-count // chunk) if count else 1
    absum = np.abs(V[:, None] * np.asarray(x, np.float64)).sum(0)
    return (chunk / 4 + 10 + blocks) * EPS * absum


@pytest.mark.parametrize("N,nlev,ld,dt", [(80, 137, 140, "float32"), (80, 5, 6, "float64"), (320, 137, 138, "float64"),
                                          (16, 1, 1, "float32"), (320, 9, 16, "bfloat16")])
def test_against_the_oracle(torch, pfvm, omesh, N, nlev, ld, dt):
    fvm = pfvm(N)
    m = omesh(N)
    V = m.dual()["V"]
    g = m.grid()
    f = synthetic.level_scalar(g["lon"], g["lat_node"], nlev)
    t = torch.from_numpy(synthetic.padded(f, ld)).cuda().to(getattr(torch, dt))
    got = fvm.integral(t, nlev).cpu().numpy()
    xs = t[:, :nlev].double().cpu().numpy()  # the values the GPU summed
    want = oracle.integral(V, xs)
    assert np.all(np.abs(got - want) <= _bound(torch, V, xs, V.shape[0])), (got - want)


def test_special_values_are_widened_exactly(torch, pfvm, omesh):
    """FP32 inputs with zeros, subnormals, the extremes of the normal range
    and both signs: every value enters the FP64 sum exactly."""
    fvm = pfvm(16)
    V = omesh(16).dual()["V"]
    rng = np.random.default_rng(9)
    vals = np.array([0.0, -0.0, 1e-40, -3e-42, 1.1754944e-38, 3.4e38, -3.4e38, 1.0, -1.5, 2.0 ** -126,
                     np.float32(np.pi)], dtype=np.float32)
    x = rng.choice(vals, size=(fvm.nnodes, 3)).astype(np.float32)
    x[:, 2] = rng.standard_normal(fvm.nnodes).astype(np.float32) * np.float32(1e-30)
    t = torch.from_numpy(synthetic.padded(x, 4)).cuda()
    got = fvm.integral(t, 3).cpu().numpy()
    want = oracle.integral(V, x)
    assert np.all(np.abs(got - want) <= _bound(torch, V, x.astype(np.float64), fvm.nnodes))


def test_conservation_of_divergence_and_curl(torch, pfvm):
    """FP64 divergence and curl of random fields: their volume-weighted sums
    over the closed sphere vanish to rounding (the oracle's pin, now on the
    GPU path end to end)."""
    fvm = pfvm(80)
    V = fvm.arrays()["V"]
    gen = torch.Generator(device="cuda").manual_seed(11)
    u, v = (torch.randn((fvm.nnodes, 8), generator=gen, device="cuda", dtype=torch.float64) for _ in range(2))
    for out in (fvm.divergence(u, v), fvm.curl(u, v)):
        I = fvm.integral(out).cpu().numpy()
        scale = np.abs(V[:, None] * out.cpu().numpy()).sum(0)
        assert np.all(np.abs(I) <= 1e-12 * scale), I / scale


def test_node_ranges_partitions_and_empty(torch, pfvm, omesh):
    from paper_1908_07038_gb300.partition import Partition
    fvm = pfvm(80)
    V = omesh(80).dual()["V"]
    gen = torch.Generator(device="cuda").manual_seed(12)
    x = torch.randn((fvm.nnodes, 12), generator=gen, device="cuda", dtype=torch.float64)
    xs = x.cpu().numpy()
    for node0, count in [(0, fvm.nnodes), (1000, 777), (fvm.nnodes - 5, 5), (321, 0)]:
        got = fvm.integral(x[node0:node0 + count] if count else x[node0:node0 + 1], node0=node0, count=count)
        got = got.cpu().numpy()
        want = oracle.integral(V[node0:node0 + count], xs[node0:node0 + count]) if count else np.zeros(12)
        b = _bound(torch, V[node0:node0 + count], xs[node0:node0 + count], count) if count else np.zeros(12)
        assert np.all(np.abs(got - want) <= b)
    whole = oracle.integral(V, xs)
    parts = np.zeros(12)
    for k in range(3):
        p = Partition(fvm, 3, k, 1)
        own = x[p.own0:p.own1]
        parts += p.integral(own, reduce=False).cpu().numpy()
        p.close()
    assert np.all(np.abs(parts - whole) <= 4 * _bound(torch, V, xs, fvm.nnodes))
