"""Posterior mean and variance of equal-size FP32-transform digital nets (n = 2^10 .. 2^18), which run the
double-float kernels, against the dense oracle: mean-only and mean + variance calls, ragged query
counts, one task, d > 8 and per-task noise.  Tolerance: |delta| within 1e-5 of the largest prior variance
R_tt Q(x, x), the FP32-transform tolerance of the posterior."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import dense  # noqa: E402
from paper_2603_16014_gb300 import inputs  # noqa: E402

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_16014_gb300 import build
    build.build()


def _run(d, T, m, nq, seed, noise_per_task=False):
    from paper_2603_16014_gb300.mtgp import MTGP
    p = inputs.make_problem("dnet", d, (m,) * T, seed=seed, eta=0.6, v=0.1, sigma2=1e-4,
                            recipe="walshcos32", mmax=m)
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    s2 = np.array([1e-4, 4e-4, 2e-3, 5e-5][:T]) if noise_per_task else p.sigma2
    Xq, xq, tq = inputs.query_points(nq, d, seed=seed + 1, tasks=T)
    mean_ref, var_ref, prior = dense.posterior(p.kind, X, y, p.eta, p.W, p.v, s2, Xq, tq)
    model = MTGP.from_problem(p, "fp32", noise_per_task=noise_per_task)
    model.set_y(torch.from_numpy(y))
    model.profile(True)
    mean_only, _ = model.posterior(p.eta, p.W, p.v, s2, torch.from_numpy(xq), torch.from_numpy(tq), variance=False)
    mean, var = model.posterior(p.eta, p.W, p.v, s2, torch.from_numpy(xq), torch.from_numpy(tq), variance=True)
    model.sync()
    prof = model.profile_read()
    model.close()
    return (mean_only.cpu().numpy(), mean.cpu().numpy(), var.cpu().numpy(), mean_ref, var_ref, prior, prof)


@pytest.mark.parametrize("d,T,m,nq", [(3, 2, 10, 37), (9, 3, 10, 5), (2, 1, 11, 64), (5, 4, 10, 129), (16, 2, 10, 3)])
def test_posterior_df_vs_dense_oracle(d, T, m, nq):
    mean_only, mean, var, mean_ref, var_ref, prior, prof = _run(d, T, m, nq, seed=71 + d)
    # the double-float path ran: rows and quadratic forms, no separate FP64 transform of the rows
    assert "var_rows" in prof and "var_quad" in prof and "var_xform" not in prof
    scale = TOL * prior.max()
    assert np.all(np.abs(mean_only - mean_ref) <= scale), np.abs(mean_only - mean_ref).max() / prior.max()
    assert np.all(np.abs(mean - mean_ref) <= scale), np.abs(mean - mean_ref).max() / prior.max()
    assert np.all(np.abs(var - var_ref) <= scale), np.abs(var - var_ref).max() / prior.max()
    # the two routes to the mean (mean-only slices, rows of the variance pass) agree far below the tolerance
    assert np.all(np.abs(mean_only - mean) <= 1e-9 * prior.max())


def test_posterior_df_per_task_noise():
    mean_only, mean, var, mean_ref, var_ref, prior, prof = _run(3, 3, 10, 23, seed=91, noise_per_task=True)
    assert "var_quad" in prof and "var_xform" not in prof
    scale = TOL * prior.max()
    assert np.all(np.abs(mean_only - mean_ref) <= scale)
    assert np.all(np.abs(mean - mean_ref) <= scale)
    assert np.all(np.abs(var - var_ref) <= scale)


@pytest.mark.parametrize("m", [12, 14, 15, 18])
def test_posterior_df_other_splits_vs_spectral_oracle(m):
    """The other register-tile splits of the double-float posterior (n = 2^12: a = 5 and 7 high bits,
    2^14: 6 and 8, 2^15: 7 and 8, 2^18: 9 and 9; 2^10, 2^11 and 2^16 are covered above), sampled mean and
    variance against the per-frequency oracle."""
    from oracle import spectral
    from paper_2603_16014_gb300.mtgp import MTGP
    d, T = 4, 2
    p = inputs.make_problem("dnet", d, (m,) * T, seed=200 + m, eta=0.6, v=0.1, sigma2=1e-4,
                            recipe="walshcos32", mmax=m)
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    Xq, xq, tq = inputs.query_points(40, d, seed=m, tasks=T)
    model = MTGP.from_problem(p, "fp32")
    model.set_y(torch.from_numpy(y))
    mean, var = model.posterior(p.eta, p.W, p.v, p.sigma2, torch.from_numpy(xq), torch.from_numpy(tq), variance=True)
    model.sync()
    model.close()
    mean, var = mean.cpu().numpy(), var.cpu().numpy()
    pick = np.array([0, 17, 39])
    mref = spectral.posterior_mean_equal(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2, Xq[pick], tq[pick])
    vref = spectral.posterior_var_equal(p.kind, p.gen, p.shift, p.m, p.eta, p.W, p.v, p.sigma2, Xq[pick], tq[pick])
    from oracle import design
    R = design.task_covariance(p.W, p.v)
    prior = np.array([R[t, t] * design.product_kernel(p.kind, Xq[i], Xq[i], p.eta) for i, t in zip(pick, tq[pick])])
    assert np.all(np.abs(mean[pick] - mref) <= TOL * prior), np.max(np.abs(mean[pick] - mref) / prior)
    assert np.all(np.abs(var[pick] - vref) <= TOL * prior), np.max(np.abs(var[pick] - vref) / prior)
