"""Seeded input generator: published SplitMix64 outputs, determinism, shapes
and the distributions the workloads state."""
import numpy as np

from paper_2601_20174_gb300 import inputs as gen


def _splitmix_ref(state, count):
    # Plain-integer SplitMix64 (Steele, Lea, Flood 2014), used only to check the
    # vectorised numpy version draws the same sequence.
    out = []
    m = (1 << 64) - 1
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & m
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_published_first_output():
    # The first output of SplitMix64 seeded with 0 is 0xE220A8397B1DCDAF
    # (reference implementation splitmix64.c by S. Vigna).
    assert _splitmix_ref(0, 1)[0] == 0xE220A8397B1DCDAF


def test_stream_matches_plain_integer_generator():
    base = gen.stream_base(123, gen.STREAM_S0)
    got = gen.splitmix64(123, gen.STREAM_S0, 50)
    assert [int(v) for v in got] == _splitmix_ref(base, 50)
    off = gen.splitmix64(123, gen.STREAM_S0, 10, offset=40)
    assert [int(v) for v in off] == _splitmix_ref(base, 50)[40:]


def test_determinism_and_stream_independence():
    a = gen.normal(7, gen.STREAM_S0, 1000)
    b = gen.normal(7, gen.STREAM_S0, 1000)
    c = gen.normal(7, gen.STREAM_RHS, 1000)
    assert np.array_equal(a, b)
    assert not np.allclose(a, c)


def test_distributions():
    u = gen.uniform(1, gen.STREAM_RHS, 200000, -1.0, 1.0)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01 and abs(u.var() - 1.0 / 3.0) < 0.01
    z = gen.normal(1, gen.STREAM_S0, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    assert abs(np.mean(z ** 4) - 3.0) < 0.05


def test_grf_covariance():
    # Empirical covariance of the separable squared-exponential field between
    # two cells at distance d approaches exp(-d^2 / (2 l^2)).
    N = 31
    fields = np.stack([gen.grf_log_kappa_2d(N, seed) for seed in range(300)])
    h = 1.0 / (N + 1)
    var = fields[:, 16, 16].var()
    assert abs(var - 1.0) < 0.2
    cov = np.mean(fields[:, 16, 16] * fields[:, 16, 19])
    assert abs(cov - np.exp(-(3 * h) ** 2 / (2 * 0.1 ** 2))) < 0.15


def test_aniso_tensor():
    t = gen.rotated_aniso_tensor(0.3, 1e-3)
    K = np.array([[t[0], t[2]], [t[2], t[1]]])
    w = np.linalg.eigvalsh(K)
    assert np.allclose(sorted(w), [1e-3, 1.0])


def test_problem_shapes():
    p = gen.poisson_2d(8, 4, 16)
    assert p.f.shape == (64, 1) and p.S0.shape == (64, 16)
    q = gen.aniso_9pt_2d(N=16, k=8, K=16, m=4)
    assert q.f.shape == (256, 4) and q.coeffs.shape == (3,)
    insts = gen.batch_instances(12, with_samples=False)
    assert all(i.N in gen.BATCH_SIDES and i.k in gen.BATCH_RANKS and i.K == 2 * i.k for i in insts)
