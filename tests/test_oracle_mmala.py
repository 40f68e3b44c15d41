"""Pins of the oracle's surrogate mMALA step (CPU only).

p1  closed-form log rho (eq:da_dino_trr_1 with rho_{0,r}) equals the direct
    Metropolis-Hastings ratio of Gaussian proposal densities and the target;
p2  linear surrogate: log rho == 0 and the chain is an exact AR(1) whose
    moments are closed-form (eq:local_gaussian is exact for a linear map);
p3  zero Jacobian: the proposal is pCN and log rho == 0 (Sec. 2.7);
p4  gradient = finite differences of the misfit; Gauss-Newton = exact Hessian
    for a linear map; Cholesky factor unique (lower, positive diagonal);
p5  full-field proposal of Prop. 5.1 has mean s m + (1-s) A~(m) and covariance
    (1-s^2) C~_post(m) of eq:surrogate_cpost;
p6  the Cholesky and eigen noise maps have the same law;
p8  r = 1: long-run chain moments equal 1-D quadrature of the target;
p9  the perturbation noise map (d_y < r) has the proposal covariance
    (1-s^2)(I+H)^-1, and with it a linear surrogate's chain is still the
    exact AR(1) of p2.
"""
import numpy as np
import pytest

from oracle import mlp, mmala, prior
from oracle.chains import OracleChains
from workloads import dis_gaussian, mlp_weights

GAMMA, DELTA = 0.1, 1.0


def _surrogate(widths, kind, seed=5, noise_var=0.05, y_seed=7):
    Ws, bs = mlp_weights(widths, seed)
    y = np.random.default_rng(y_seed).standard_normal(widths[-1])
    return mmala.Surrogate(Ws=Ws, bs=bs, act=kind, y=y, noise_var=noise_var)


@pytest.mark.parametrize("r", [1, 2, 5, 16])
@pytest.mark.parametrize("kind", [mlp.ACT_TANH, mlp.ACT_GELU])
def test_p1_closed_form_equals_direct_density_ratio(r, kind):
    sur = _surrogate([r, 12, 12, 7], kind, noise_var=0.3)
    rng = np.random.default_rng(r)
    dt = 0.7
    for _ in range(4):
        a = rng.standard_normal(r)
        geo_a = mmala.geometry(sur, a)
        _, b = mmala.reduced_proposal(a, geo_a, rng.standard_normal(r), dt)
        geo_b = mmala.geometry(sur, b)
        closed = mmala.log_rho(a, geo_a, b, geo_b, dt)
        direct = (mmala.log_target(geo_b, b) + mmala.log_q(b, geo_b, a, dt)
                  - mmala.log_target(geo_a, a) - mmala.log_q(a, geo_a, b, dt))
        assert abs(closed - direct) < 1e-9 * max(1.0, abs(direct))
        assert abs(closed) > 1e-6        # a genuinely nonlinear case


def test_p1_fails_with_the_printed_gradient_sign():
    # the reduced ppg printed as J^T (y - f) gives a ratio that is not the MH ratio
    sur = _surrogate([3, 8, 5], mlp.ACT_TANH, noise_var=0.3)
    rng = np.random.default_rng(1)
    a, b, dt = rng.standard_normal(3), rng.standard_normal(3), 0.5
    geo_a, geo_b = mmala.geometry(sur, a), mmala.geometry(sur, b)
    direct = (mmala.log_target(geo_b, b) + mmala.log_q(b, geo_b, a, dt)
              - mmala.log_target(geo_a, a) - mmala.log_q(a, geo_a, b, dt))
    flipped_a = mmala.Geometry(**{**geo_a.__dict__, "g": -geo_a.g})
    flipped_b = mmala.Geometry(**{**geo_b.__dict__, "g": -geo_b.g})
    wrong = mmala.log_rho(a, flipped_a, b, flipped_b, dt)
    assert abs(wrong - direct) > 1e-3


def test_p2_linear_surrogate_log_rho_is_zero():
    sur = _surrogate([6, 9, 4], mlp.ACT_IDENTITY, noise_var=0.02)
    rng = np.random.default_rng(2)
    for dt in (0.1, 0.5, 2.0):
        a = rng.standard_normal(6)
        b = 3 * rng.standard_normal(6)
        lr = mmala.log_rho(a, mmala.geometry(sur, a), b, mmala.geometry(sur, b), dt)
        assert abs(lr) < 1e-9


def test_p2_linear_surrogate_chain_is_exact_ar1():
    n, r = 3, 3
    sur = _surrogate([r, 5, 4], mlp.ACT_IDENTITY, noise_var=0.5)
    E, D = prior.kle_basis(n, GAMMA, DELTA, r)
    C = 4000
    dt = 0.5
    s = mmala.s_of_dt(dt)
    m0 = np.zeros(n * n)
    ch = OracleChains(sur, E, D, n, GAMMA, DELTA, C, dt, seed=31, m0=m0, noise="cholesky")
    W = sur.Ws[1] @ sur.Ws[0]
    c = sur.Ws[1] @ sur.bs[0] + sur.bs[1]
    Cpost = np.linalg.inv(np.eye(r) + W.T @ W / sur.noise_var)
    mpost = Cpost @ W.T @ (sur.y - c) / sur.noise_var
    for j in range(1, 4):
        ch.step()
        assert ch.last["accepted"].all()
        mean = mpost + s ** j * (np.zeros(r) - mpost)
        cov = (1 - s ** (2 * j)) * Cpost
        Lc = np.linalg.cholesky(cov)
        w = np.linalg.solve(Lc, (ch.m_r - mean).T).T        # should be N(0, I)
        assert np.all(np.abs(w.mean(0)) < 5 / np.sqrt(C))
        assert np.abs(np.cov(w.T) - np.eye(r)).max() < 7 / np.sqrt(C)


def test_p3_zero_jacobian_is_pcn():
    sur = _surrogate([4, 6, 3], mlp.ACT_GELU)
    sur.Ws[-1] = np.zeros_like(sur.Ws[-1])
    rng = np.random.default_rng(3)
    a, xi, dt = rng.standard_normal(4), rng.standard_normal(4), 0.8
    s = mmala.s_of_dt(dt)
    geo_a = mmala.geometry(sur, a)
    assert np.all(geo_a.g == 0) and np.all(geo_a.H == 0)
    _, b = mmala.reduced_proposal(a, geo_a, xi, dt)
    assert np.allclose(b, s * a + np.sqrt(1 - s * s) * xi, atol=1e-15)
    assert abs(mmala.log_rho(a, geo_a, b, mmala.geometry(sur, b), dt)) < 1e-14


def test_p4_gradient_is_misfit_derivative_and_cholesky_unique():
    sur = _surrogate([5, 7, 6], mlp.ACT_TANH, noise_var=0.2)
    a = np.random.default_rng(4).standard_normal(5)
    geo = mmala.geometry(sur, a)
    for k in range(5):
        e = np.zeros(5)
        e[k] = 1e-6
        fd = (mmala.geometry(sur, a + e).phi - mmala.geometry(sur, a - e).phi) / 2e-6
        assert fd == pytest.approx(geo.g[k], rel=1e-6, abs=1e-8)
    L = geo.L
    assert np.allclose(np.triu(L, 1), 0) and np.all(np.diag(L) > 0)
    assert np.linalg.norm(L @ L.T - (np.eye(5) + geo.H)) < 1e-13 * np.linalg.norm(geo.H + np.eye(5))
    assert geo.hld == pytest.approx(0.5 * np.linalg.slogdet(np.eye(5) + geo.H)[1], rel=1e-13)


def test_p4_gauss_newton_is_exact_hessian_for_linear_map():
    sur = _surrogate([4, 6, 5], mlp.ACT_IDENTITY, noise_var=0.3)
    a = np.random.default_rng(5).standard_normal(4)
    geo = mmala.geometry(sur, a)
    Hfd = np.empty((4, 4))
    for k in range(4):
        e = np.zeros(4)
        e[k] = 1e-5
        Hfd[:, k] = (mmala.geometry(sur, a + e).g - mmala.geometry(sur, a - e).g) / 2e-5
    assert np.allclose(Hfd, geo.H, rtol=1e-7, atol=1e-7)


@pytest.mark.parametrize("kind", ["kle", "dis"])
def test_p5_full_proposal_law_is_surrogate_mmala(kind):
    n, r, dt = 3, 2, 0.6
    N = n * n
    s = mmala.s_of_dt(dt)
    if kind == "kle":
        E, D = prior.kle_basis(n, GAMMA, DELTA, r)
    else:
        E, D = prior.dis_basis(n, GAMMA, DELTA, dis_gaussian(N, r, 4))
    sur = _surrogate([r, 6, 3], mlp.ACT_TANH, noise_var=0.1)
    m = prior.prior_sample(n, GAMMA, DELTA, np.random.default_rng(6).standard_normal(N))
    a = E @ m
    geo = mmala.geometry(sur, a)

    def full(xi, z):
        _, b = mmala.reduced_proposal(a, geo, xi, dt)
        M = prior.prior_sample(n, GAMMA, DELTA, z)
        return mmala.field_proposal(m, b, M, E, D, dt)

    mean = full(np.zeros(r), np.zeros(N))
    cols = [full(np.eye(r)[i], np.zeros(N)) - mean for i in range(r)]
    cols += [full(np.zeros(r), np.eye(N)[q]) - mean for q in range(N)]
    T = np.array(cols).T
    cov = T @ T.T
    # the paper's quantities (Sec. 5.2-5.3): eigen-decomposition H = P diag(d) P^T
    d, P = np.linalg.eigh(geo.H)
    A = prior.prior_operator(n, GAMMA, DELTA).toarray()
    Cpr = np.linalg.inv(A @ A)
    Psi_t = D @ P
    Psi_t_star = P.T @ E
    Cpost = Cpr - Psi_t @ np.diag(d / (d + 1)) @ Psi_t_star @ Cpr
    A_tilde = Psi_t @ np.diag(d / (d + 1)) @ Psi_t_star @ m - Psi_t @ np.diag(1 / (d + 1)) @ P.T @ geo.g
    assert np.allclose(mean, s * m + (1 - s) * A_tilde, atol=1e-12)
    assert np.allclose(cov, (1 - s * s) * Cpost, atol=1e-12 * np.abs(Cpost).max())


def test_p6_cholesky_and_eigen_maps_have_the_same_law():
    r, dt = 4, 0.5
    sur = _surrogate([r, 8, 6], mlp.ACT_GELU, noise_var=0.1)
    a = np.random.default_rng(7).standard_normal(r)
    geo = mmala.geometry(sur, a)
    chol0 = mmala.reduced_proposal(a, geo, np.zeros(r), dt)[1]
    eig0 = mmala.reduced_proposal_eigen(a, geo.H, geo.g, np.zeros(r), dt)
    assert np.allclose(chol0, eig0, atol=1e-12)
    Tc = np.array([mmala.reduced_proposal(a, geo, e, dt)[1] - chol0 for e in np.eye(r)]).T
    Te = np.array([mmala.reduced_proposal_eigen(a, geo.H, geo.g, e, dt) - eig0 for e in np.eye(r)]).T
    assert np.allclose(Tc @ Tc.T, Te @ Te.T, atol=1e-12)


def test_accept_rule_edges():
    lu = np.log(np.array([0.5, 0.5, 0.5, 0.5, 0.5]))
    lr = np.array([np.nan, 0.0, np.log(0.5), np.log(0.5) - 1e-12, np.inf])
    assert list(mmala.accept(lu, lr)) == [False, True, True, False, False]


def test_p8_r1_chain_moments_match_quadrature():
    n, r, dt = 3, 1, 1.0
    sur = _surrogate([1, 8, 2], mlp.ACT_TANH, seed=11, noise_var=0.25, y_seed=12)
    E, D = prior.kle_basis(n, GAMMA, DELTA, r)
    x = np.linspace(-9, 9, 36001)
    geo = mmala.geometry(sur, x[:, None])
    logp = -geo.phi - 0.5 * x * x
    p = np.exp(logp - logp.max())
    p /= np.trapezoid(p, x)
    mean_q = np.trapezoid(x * p, x)
    var_q = np.trapezoid((x - mean_q) ** 2 * p, x)
    C = 3000
    ch = OracleChains(sur, E, D, n, GAMMA, DELTA, C, dt, seed=77, noise="cholesky")
    ch.step(60)
    acc = []
    samples = []
    for _ in range(60):
        ch.step()
        acc.append(ch.last["accepted"].mean())
        samples.append(ch.m_r[:, 0].copy())
    S = np.array(samples)
    assert 0.2 < np.mean(acc) < 1.0
    sd = np.sqrt(var_q)
    # final ensemble: C independent draws
    assert abs(S[-1].mean() - mean_q) < 5 * sd / np.sqrt(C)
    assert abs(S.mean() - mean_q) < 5 * sd / np.sqrt(C)
    assert abs(S.var() / var_q - 1) < 0.06


def test_p9_perturbation_map_has_the_proposal_covariance():
    r, dy, dt, nv = 7, 3, 0.5, 0.1
    s = mmala.s_of_dt(dt)
    sur = _surrogate([r, 8, dy], mlp.ACT_TANH, noise_var=nv)
    a = np.random.default_rng(8).standard_normal(r)
    geo = mmala.geometry(sur, a)
    mu, b0 = mmala.reduced_proposal_perturbation(a, geo, np.zeros(r), np.zeros(dy), nv, dt)
    assert np.allclose(b0, mu, atol=1e-13) and np.allclose(mu, mmala.proposal_mean(a, geo, dt))
    cols = [mmala.reduced_proposal_perturbation(a, geo, e[:r], e[r:], nv, dt)[1] - b0
            for e in np.eye(r + dy)]
    T = np.array(cols).T                                   # b - mu = T [xi1; xi2]
    cov_ref = (1 - s * s) * np.linalg.inv(np.eye(r) + geo.J.T @ geo.J / nv)
    assert np.allclose(T @ T.T, cov_ref, atol=1e-12 * np.abs(cov_ref).max())
    # dropping the observation-space normals (or mis-scaling K) breaks the law
    T1 = T[:, :r]
    assert np.abs(T1 @ T1.T - cov_ref).max() > 1e-3 * np.abs(cov_ref).max()


def test_p9_perturbation_chain_is_exact_ar1_for_linear_surrogate():
    n, r, dy = 3, 5, 2
    sur = _surrogate([r, 4, dy], mlp.ACT_IDENTITY, noise_var=0.3)
    E, D = prior.kle_basis(n, GAMMA, DELTA, r)
    C, dt = 4000, 0.5
    s = mmala.s_of_dt(dt)
    ch = OracleChains(sur, E, D, n, GAMMA, DELTA, C, dt, seed=32, m0=np.zeros(n * n),
                      noise="perturbation")
    W = sur.Ws[1] @ sur.Ws[0]
    c = sur.Ws[1] @ sur.bs[0] + sur.bs[1]
    Cpost = np.linalg.inv(np.eye(r) + W.T @ W / sur.noise_var)
    mpost = Cpost @ W.T @ (sur.y - c) / sur.noise_var
    for j in range(1, 4):
        ch.step()
        assert ch.last["accepted"].all()
        mean = mpost + s ** j * (np.zeros(r) - mpost)
        cov = (1 - s ** (2 * j)) * Cpost
        w = np.linalg.solve(np.linalg.cholesky(cov), (ch.m_r - mean).T).T
        assert np.all(np.abs(w.mean(0)) < 5 / np.sqrt(C))
        assert np.abs(np.cov(w.T) - np.eye(r)).max() < 7 / np.sqrt(C)


def test_given_noise_reproduces_the_philox_step():
    """Feeding a step the arrays the chain would draw itself changes nothing;
    feeding other arrays changes the proposal."""
    from oracle import philox
    n, r, dy = 3, 5, 2
    sur = _surrogate([r, 4, dy], mlp.ACT_TANH, noise_var=0.3)
    E, D = prior.kle_basis(n, GAMMA, DELTA, r)
    C, dt = 6, 0.3
    for noise in ("cholesky", "perturbation"):
        a = OracleChains(sur, E, D, n, GAMMA, DELTA, C, dt, seed=5, noise=noise)
        b = OracleChains(sur, E, D, n, GAMMA, DELTA, C, dt, seed=5, noise=noise)
        ids = np.arange(C, dtype=np.uint64)
        given = dict(xi=philox.normals(5, philox.STREAM_XI, 0, ids, r),
                     xi2=philox.normals(5, philox.STREAM_XI2, 0, ids, dy),
                     z=philox.normals(5, philox.STREAM_Z, 0, ids, n * n),
                     log_u=np.log(philox.uniform(5, philox.STREAM_U, 0, ids)))
        a.step()
        b.step(noise=given)
        for k in ("b", "log_rho", "log_u", "m_new"):
            assert np.array_equal(a.last[k], b.last[k]), k
        b.step(noise=dict(xi=np.zeros((C, r))))
        a.step()
        assert not np.allclose(a.last["b"], b.last["b"])
    with pytest.raises(ValueError):
        OracleChains(sur, E, D, n, GAMMA, DELTA, C, dt, seed=5, noise="auto")


def test_eigen_map_law_and_the_papers_form():
    """The symmetric eigen map has covariance (1 - s^2)(I + H)^-1 exactly, and
    equals the paper's P diag(sqrt((1 - s^2)/(d + 1))) Xi of
    eq:reduced_space_sampling for Xi = P^T xi."""
    r, dt = 6, 0.4
    s = mmala.s_of_dt(dt)
    sur = _surrogate([r, 9, 4], mlp.ACT_GELU, noise_var=0.2)
    a = np.random.default_rng(12).standard_normal(r)
    geo = mmala.geometry(sur, a)
    mu, b0 = mmala.reduced_proposal_sqrt(a, geo, np.zeros(r), dt)
    assert np.allclose(b0, mu, atol=1e-14)
    T = np.array([mmala.reduced_proposal_sqrt(a, geo, e, dt)[1] - b0 for e in np.eye(r)]).T
    cov = (1 - s * s) * np.linalg.inv(np.eye(r) + geo.H)
    assert np.allclose(T @ T.T, cov, atol=1e-12 * np.abs(cov).max())
    assert np.allclose(T, T.T, atol=1e-13)                # a symmetric root
    xi = np.random.default_rng(13).standard_normal(r)
    d, P = np.linalg.eigh(geo.H)
    paper = mmala.reduced_proposal_eigen(a, geo.H, geo.g, P.T @ xi, dt)
    assert np.allclose(mmala.reduced_proposal_sqrt(a, geo, xi, dt)[1], paper, atol=1e-12)
