"""The Gauss-Newton update on the GPU (gsdf_gn_update: the FP64 solve of the damped normal
equations and the left update T <- exp(xi^) T of Sec. 4.1, the last stage of every tracking
step) against the oracle's Cholesky solve and exponential map, on systems whose conditioning,
scaling and degeneracy are chosen.  Bars:
  * degenerate exactly when the oracle's Cholesky factorisation fails its pivot test (the
    systems keep their smallest relative pivot 6x or more away from the 1e-12 threshold);
  * |xi - xi_oracle| <= max(1e-13, 2e-14 kappa) max|xi_oracle| for condition number kappa of the
    diagonally scaled matrix: both are backward-stable FP64 solves, whose forward errors are of
    order kappa times the unit roundoff;
  * the pose equals exp(xi^) T evaluated by the oracle at the device's own xi within 1e-13, and
    a degenerate system leaves it unchanged bit for bit with xi = 0.
"""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_13652_gb300 import gsdf

    gsdf.load_library()
    return gsdf


def _hb(H, b):
    return np.concatenate([[H[i, j] for i in range(6) for j in range(i, 6)], b])


def _poses(rng, n):
    return np.stack([O.se3_exp(np.concatenate([rng.normal(0, 0.7, 3), rng.normal(0, 1.5, 3)])) for _ in range(n)])


def _run(G, Hb, n_valid, damping, T):
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    n = len(Hb)
    Tt = d(T)
    xi = torch.full((n, 6), np.nan, dtype=torch.float64, device="cuda")
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    G.gn_update(d(Hb), d(np.asarray(n_valid, np.int64)), damping, Tt, xi, st)
    torch.cuda.synchronize()
    return Tt.cpu().numpy(), xi.cpu().numpy(), st.cpu().numpy()


def _check(G, Hb, n_valid, damping, T, kappa):
    Tn, xi, st = _run(G, Hb, n_valid, damping, T)
    n_bad = 0
    for s in range(len(Hb)):
        bad, xo = O.solve6(Hb[s, :21], Hb[s, 21:], damping, int(n_valid[s]))
        assert (st[s] != 0) == bool(bad), (s, st[s], bad)
        if bad:
            n_bad += 1
            assert st[s] == G.GSDF_ERR_DEGENERATE
            assert np.array_equal(Tn[s], T[s]) and not xi[s].any()
            continue
        tol = max(1e-13, 2e-14 * kappa[s]) * np.abs(xo).max()
        assert np.abs(xi[s] - xo).max() <= tol, (s, kappa[s], np.abs(xi[s] - xo).max() / np.abs(xo).max())
        ref = O.se3_exp(xi[s]) @ T[s]
        assert np.abs(Tn[s] - ref).max() <= 1e-13, (s, np.abs(Tn[s] - ref).max())
        assert np.array_equal(Tn[s][3], [0.0, 0.0, 0.0, 1.0])
    return Tn, xi, st, n_bad


@pytest.mark.parametrize("damping", [0.0, 1e-4])
def test_conditioned_and_scaled_systems(G, damping):
    """2000 SPD systems H = S Q diag(lam) Q^T S, lam log-spaced over kappa in 1 .. 1e6, row and
    column scales S in 10^[-1, 1] (rotation and translation units differ), xi ~ 1e-3."""
    rng = np.random.default_rng(11)
    n = 2000
    kappas = np.array([1.0, 1e2, 1e4, 1e6])[np.arange(n) % 4]
    Hb = np.zeros((n, 27))
    for s in range(n):
        Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
        S = np.diag(10.0 ** rng.uniform(-1, 1, 6))
        H = S @ (Q * np.logspace(0, np.log10(kappas[s]), 6)) @ Q.T @ S * 10.0 ** rng.uniform(-3, 6)
        xt = rng.normal(0, 1e-3, 6)
        Hb[s] = _hb(H, -(H @ xt))
    _, _, _, n_bad = _check(G, Hb, np.full(n, 1000), damping, _poses(rng, n), kappas)
    assert n_bad == 0


@pytest.mark.parametrize("damping", [0.0, 1e-4])
def test_pivot_test_matches_cholesky(G, damping):
    """H = L D L^T with one pivot delta in {1e-8, 1e-10, 1e-14, 1e-16} at each position j, the other
    pivots in [0.5, 2] and L unit lower triangular with N(0, 0.3) entries (diagonal entries of H
    between 0.5 and ~16): without damping the 1e-12 test keeps the first two and rejects the last
    two (margins >= 6x and >= 50x), wherever the small pivot sits; with damping all are solvable."""
    rng = np.random.default_rng(12)
    Hb, kappa = [], []
    for delta in (1e-8, 1e-10, 1e-14, 1e-16):
        for j in range(6):
            for _ in range(4):
                L = np.eye(6) + np.tril(rng.normal(0, 0.3, (6, 6)), -1)
                d = rng.uniform(0.5, 2.0, 6)
                d[j] = delta
                H = L @ np.diag(d) @ L.T
                Hb.append(_hb(H, -(H @ rng.normal(0, 1e-3, 6))))  # increments ~1e-3, as in tracking
                kappa.append(1.0 / max(delta, damping))
    Hb = np.array(Hb)
    _, _, st, n_bad = _check(G, Hb, np.full(len(Hb), 500), damping, _poses(rng, len(Hb)), np.array(kappa) * 100)
    if damping == 0.0:
        assert n_bad == len(Hb) // 2  # exactly the 1e-14 and 1e-16 halves
        assert not st[: len(Hb) // 2].any() and st[len(Hb) // 2:].all()
    else:
        assert n_bad == 0


def test_rank_deficient_and_invalid_systems(G):
    rng = np.random.default_rng(13)
    A, B = rng.normal(size=(50, 3)), rng.normal(size=(3, 6))
    J = A @ B  # rank 3: the geometry of a single plane
    H = J.T @ J
    b = J.T @ rng.normal(size=50)
    good = np.diag([4.0, 3.0, 2.0, 5.0, 6.0, 7.0]) + 0.1
    cases = [
        (_hb(H, b), 1000),                                       # rank deficient
        (_hb(good, np.ones(6) * 1e-3), 5),                        # fewer than 6 residuals
        (_hb(good - np.diag([0, 0, 0, 0, 0, good[5, 5]]), np.ones(6)), 1000),   # zero diagonal entry
        (_hb(good - np.diag([0, 0, 2 * good[2, 2], 0, 0, 0]), np.ones(6)), 1000),  # negative diagonal entry
        (_hb(np.zeros((6, 6)), np.zeros(6)), 1000),               # nothing observed
        (_hb(good, np.ones(6) * 1e-3), 1000),                     # a well-posed one among them
    ]
    nan_diag = _hb(good, np.ones(6))
    nan_diag[6] = np.nan  # H_11
    cases.append((nan_diag, 1000))
    Hb = np.array([c[0] for c in cases])
    nv = np.array([c[1] for c in cases])
    T = _poses(rng, len(Hb))
    Tn, xi, st = _run(G, Hb, nv, 0.0, T)
    assert list(st != 0) == [True, True, True, True, True, False, True]
    for s in range(len(Hb)):
        if st[s]:
            assert np.array_equal(Tn[s], T[s]) and not xi[s].any()
    bad, xo = O.solve6(Hb[5, :21], Hb[5, 21:], 0.0, 1000)
    assert not bad and np.abs(xi[5] - xo).max() <= 1e-13 * np.abs(xo).max()
    assert O.solve6(Hb[0, :21], Hb[0, 21:], 0.0, 1000)[0]  # the oracle agrees on the plane
    # with damping the plane's system is solvable (kappa ~ 1 / (1e-4 / 6))
    _check(G, Hb[:1], nv[:1], 1e-4, T[:1], np.array([1e6]))


def test_values_outside_the_normal_range(G):
    """Subnormal entries (an off-diagonal term, a gradient component) and a matrix near the top of
    the FP64 range: the powers of two of the warp-parallel solve would leave the normal range, so
    the update takes its serial path; it must agree with the oracle like the others."""
    rng = np.random.default_rng(15)
    base = np.diag([4.0, 3.0, 2.0, 5.0, 6.0, 7.0]) + 0.1
    Hs, bs = [], []
    H = base.copy()
    H[0, 1] = H[1, 0] = 3e-310
    Hs.append(H)
    bs.append(-(H @ rng.normal(0, 1e-3, 6)))
    H = base.copy()
    Hs.append(H)
    b = -(H @ rng.normal(0, 1e-3, 6))
    b[4] = 5e-311
    bs.append(b)
    H = base * 1e300
    Hs.append(H)
    bs.append(-(H @ rng.normal(0, 1e-3, 6)))
    H = base * 1e-300
    Hs.append(H)
    bs.append(-(H @ rng.normal(0, 1e-3, 6)))
    Hb = np.array([_hb(H, b) for H, b in zip(Hs, bs)])
    for damping in (0.0, 1e-4):
        _, _, _, n_bad = _check(G, Hb, np.full(len(Hb), 100), damping, _poses(rng, len(Hb)), np.full(len(Hb), 10.0))
        assert n_bad == 0


def test_exponential_map_regimes(G):
    """H = h I and b = -h xi make xi the increment; rotation angles on both sides of the series
    threshold th^2 = 1e-2 and far beyond it, rotations stay orthonormal."""
    rng = np.random.default_rng(14)
    angles = [0.0, 1e-9, 1e-4, 0.05, 0.0999, 0.1001, 0.5, 3.0]
    Hb, xts = [], []
    for k, th in enumerate(angles):
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        xt = np.concatenate([axis * th, rng.normal(0, 0.2, 3)])
        h = 10.0 ** (k - 3)
        Hb.append(_hb(np.eye(6) * h, -h * xt))
        xts.append(xt)
    Hb, xts = np.array(Hb), np.array(xts)
    T = _poses(rng, len(Hb))
    Tn, xi, st, n_bad = _check(G, Hb, np.full(len(Hb), 100), 0.0, T, np.ones(len(Hb)))
    assert n_bad == 0
    assert np.abs(xi - xts).max() <= 1e-15 * np.abs(xts).max()
    for s in range(len(Hb)):
        R = Tn[s][:3, :3]
        assert np.abs(R.T @ R - np.eye(3)).max() <= 1e-14
