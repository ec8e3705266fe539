"""The seeded synthetic workloads: reproducible, and distributed as their recipes say."""
import numpy as np

import workloads


def test_splitmix64_reference_values():
    # splitmix64 from state 0: the first outputs of the published generator
    z = workloads.splitmix64_stream(0, 3)
    assert [int(x) for x in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_gaussian_stream_moments():
    g = workloads.gaussian_stream(123, 400000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1.0) < 0.01


def test_batch_problem_set():
    b = workloads.batch_problems()
    assert len(b) == 512 and b == workloads.batch_problems()
    nx = np.array([p["Nx"] for p in b])
    assert nx.min() >= 64 and nx.max() <= 2048
    # log-uniform: the median side is near sqrt(64 * 2048) = 362
    assert 250 < np.median(nx) < 520
    assert {p["st"] for p in b} == {5, 9} and all(p["tol"] == 1e-8 for p in b)


def test_request_stream():
    r = workloads.request_stream()
    assert len(r) == 10000
    t = np.array([x["t_arrival"] for x in r])
    gaps = np.diff(t)
    assert np.all(gaps >= 0) and abs(gaps.mean() - 0.5e-3) < 0.03e-3
    assert {x["st"] for x in r} == {5, 9, 17} and {x["tol"] for x in r} == {1e-6, 1e-10}
    side = np.array([x["Nx"] for x in r])
    assert side.min() >= 32 and side.max() <= 8192


def test_smooth_rhs_is_a_sum_of_its_modes():
    Nx, Ny = 37, 29
    k, l, a = workloads.smooth_random_modes(Nx, Ny, 5, kmax=20)
    f = workloads.smooth_random_rhs(Nx, Ny, 5, kmax=20)
    i = np.arange(1, Nx + 1)
    j = np.arange(1, Ny + 1)
    ref = sum(aa * np.outer(np.sin(ll * np.pi * j / (Ny + 1)), np.sin(kk * np.pi * i / (Nx + 1)))
              for kk, ll, aa in zip(k, l, a))
    np.testing.assert_allclose(f, ref, atol=1e-12)
    assert np.all(k * k + l * l <= 400)
