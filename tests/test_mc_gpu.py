"""Batched Monte-Carlo (mc_solve_batch, Sec. 5 and Algorithm 1 of the paper)
against the oracle: every GPU path equals the oracle's pathwise solution (an
SG problem with one mode whose coefficient and manufactured solution are
evaluated at the sample), the returned statistics equal the sample mean and
the unbiased sample variance of those paths (eqs. mc-mean-estimator,
mc-variance-estimator-unbiased), and with many samples the mean lies within a
few standard errors of the exact mean."""
import numpy as np
import pytest

import paper_2605_21046_gb300 as sg
from paper_2605_21046_gb300 import inputs as I
from oracle import hermite, manufactured, operator

from test_march_gpu import to_product

pytestmark = pytest.mark.gpu


def shared_phi_exact(M, q, eta=0.35, T=(0.0, 1.0, 1.0)):
    idx = hermite.multi_indices(M, q)
    c = [1.0 if not any(a) else eta ** int(sum(a)) for a in idx]
    return {"q": q, "c": c, "phi": [[("sin", 1), ("sin", 1)] for _ in idx], "T": list(T)}


def pathwise(spec, exact, xi):
    """The oracle's pathwise problem for one sample."""
    idx_q = hermite.multi_indices(spec["M"], exact["q"])
    g = sum(c * hermite.Psi(a, xi) for c, a in zip(exact["c"], idx_q))
    coef = []
    for p in spec["coef"]:
        p = dict(p)
        p["amp"] = float(p["amp"]) * float(hermite.Psi(p["mu"], xi))
        p["mu"] = (0,)
        coef.append(p)
    s = dict(spec, M=1, P=0, coef=coef)
    return s, {"q": 0, "c": [float(g)], "phi": [exact["phi"][0]], "T": exact["T"]}


def test_paths_and_statistics_match_oracle(cuda):
    torch = cuda
    spec = dict(I.config_small_2d_q1(), n_slabs=10)
    exact = shared_phi_exact(2, 2)
    xi = np.random.default_rng(4096).standard_normal((7, 2))
    slabs = 3
    spec_run = dict(spec, n_slabs=slabs, T=slabs * spec["T"] / spec["n_slabs"])
    ctx = sg.sg_setup_spec(spec_run)
    sg.sg_set_exact(ctx, to_product(exact))
    mean, var, paths, st = sg.mc_solve_batch(ctx, xi, batch=3, mg_precision=sg.SG_PREC_FP64, rtol=1e-12,
                                             keep_paths=True)
    n_x, n_t = ctx.info["n_x"], ctx.info["n_t"]
    ctx.destroy()
    assert st["batches"] == 1 and st["n_samples"] == 7 and st["max_rel_residual"] <= 1e-12
    P = paths.cpu().numpy().reshape(7, n_t, n_x)
    finals = []
    for s in range(7):
        sp, ex = pathwise(spec_run, exact, xi[s])
        p = operator.SGProblem(sp)
        U = manufactured.Manufactured(p, ex).march(slabs)[-1]
        assert np.abs(P[s] - U[0]).max() <= 1e-8 * np.abs(U).max(), s
        finals.append(U[0, -1])
    finals = np.array(finals)
    assert np.abs(mean.cpu().numpy() - finals.mean(axis=0)).max() <= 1e-9 * np.abs(finals).max()
    assert np.abs(var.cpu().numpy() - finals.var(axis=0, ddof=1)).max() <= 1e-9 * finals.var(axis=0, ddof=1).max()


@pytest.mark.parametrize("tile", [1, 4, 64])
def test_two_meshes_in_one_system_match_oracle(cuda, tile):
    """mc_solve_meshes: samples on an 8x8 Q1 and a 6x10 Q1 mesh (and a 3D
    4x4x4 Q1 case below) share one system per slab and one apply launch;
    every path equals the oracle's pathwise solution on its own mesh."""
    torch = cuda
    base = dict(I.config_small_2d_q1(), n_slabs=10)
    slabs = 3
    specs = [dict(base, n_slabs=slabs, T=slabs * base["T"] / base["n_slabs"]),
             dict(base, cells=(6, 10), n_slabs=slabs, T=slabs * base["T"] / base["n_slabs"])]
    exact = shared_phi_exact(2, 2)
    xis = [np.random.default_rng(21).standard_normal((5, 2)), np.random.default_rng(22).standard_normal((3, 2))]
    ctxs = []
    for sp in specs:
        c = sg.sg_setup_spec(sp)
        sg.sg_set_exact(c, to_product(exact))
        ctxs.append(c)
    means, vars_, paths, st = sg.mc_solve_meshes(ctxs, xis, tile=tile, mg_precision=sg.SG_PREC_FP64, rtol=1e-12,
                                                 keep_paths=True)
    infos = [c.info for c in ctxs]
    for c in ctxs:
        c.destroy()
    assert st["n_samples"] == 8 and st["max_rel_residual"] <= 1e-12
    for sp, xi, info, mean, var, path in zip(specs, xis, infos, means, vars_, paths):
        n_t, n_x = info["n_t"], info["n_x"]
        Pp = path.cpu().numpy().reshape(xi.shape[0], n_t, n_x)
        finals = []
        for s_ in range(xi.shape[0]):
            psp, ex = pathwise(sp, exact, xi[s_])
            U = manufactured.Manufactured(operator.SGProblem(psp), ex).march(slabs)[-1]
            assert np.abs(Pp[s_] - U[0]).max() <= 1e-8 * np.abs(U).max()
            finals.append(U[0, -1])
        finals = np.array(finals)
        assert np.abs(mean.cpu().numpy() - finals.mean(axis=0)).max() <= 1e-9 * np.abs(finals).max()
        assert np.abs(var.cpu().numpy() - finals.var(axis=0, ddof=1)).max() <= 1e-9 * finals.var(axis=0, ddof=1).max()


def test_paths_3d_match_oracle(cuda):
    torch = cuda
    spec = dict(dim=3, cells=(4, 4, 4), lo=(0.0,) * 3, hi=(1.0,) * 3, k=1, r=1, n_slabs=2, T=0.2, M=2, P=1,
                coef=I.linear_sine_coef(2, 3, 0.08, [(1, 1, 1), (2, 1, 1)]))
    exact = {"q": 1, "c": [1.0, 0.3, 0.2], "phi": [[("sin", 1)] * 3] * 3, "T": [0.0, 1.0, 1.0]}
    xi = np.random.default_rng(31).standard_normal((3, 2))
    ctx = sg.sg_setup_spec(spec)
    sg.sg_set_exact(ctx, to_product(exact))
    mean, var, paths, st = sg.mc_solve_batch(ctx, xi, batch=2, mg_precision=sg.SG_PREC_FP32, rtol=1e-12,
                                             keep_paths=True)
    n_t, n_x = ctx.info["n_t"], ctx.info["n_x"]
    ctx.destroy()
    P = paths.cpu().numpy().reshape(3, n_t, n_x)
    for s_ in range(3):
        psp, ex = pathwise(spec, exact, xi[s_])
        U = manufactured.Manufactured(operator.SGProblem(psp), ex).march(2)[-1]
        assert np.abs(P[s_] - U[0]).max() <= 1e-8 * np.abs(U).max()


def test_more_samples_than_one_tile_family(cuda):
    """600 samples (beyond one Vanka tile of 64 and many apply tiles) in one
    system: the converged statistics stay within sampling error of the exact
    mean, and every slab reaches the tolerance."""
    spec = dict(I.config_small_2d_q1(), cells=(8, 8), n_slabs=4, T=1.0)
    exact = shared_phi_exact(2, 2, T=(0.0, 1.0))
    N = 600
    xi = np.random.default_rng(41).standard_normal((N, 2))
    ctx = sg.sg_setup_spec(spec)
    sg.sg_set_exact(ctx, to_product(exact))
    mean, var, _, st = sg.mc_solve_batch(ctx, xi, batch=64, mg_precision=sg.SG_PREC_BF16, rtol=1e-10)
    ctx.destroy()
    mesh = operator.space_fe.Mesh(2, spec["cells"], spec["lo"], spec["hi"], spec["k"])
    X = mesh.node_coords()
    phi = np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])
    c = np.array(exact["c"])
    se = np.sqrt((c[1:] ** 2).sum() * phi.max() ** 2 / N)
    assert np.abs(mean.cpu().numpy() - c[0] * phi).max() <= 4 * se + 5e-3
    assert st["max_rel_residual"] <= 1e-10 and st["batches"] == 1
    assert 8 <= st["tile"] <= 64 and st["chunk"] >= 1          # the autotuned apply shape


def test_mean_within_standard_errors_of_exact(cuda):
    spec = dict(I.config_small_2d_q1(), cells=(16, 16), k=2, n_slabs=4, T=1.0)
    exact = shared_phi_exact(2, 2, T=(0.0, 1.0))
    N = 512
    xi = np.random.default_rng(7).standard_normal((N, 2))
    ctx = sg.sg_setup_spec(spec)
    sg.sg_set_exact(ctx, to_product(exact))
    mean, var, _, st = sg.mc_solve_batch(ctx, xi, batch=256, mg_precision=sg.SG_PREC_FP32, rtol=1e-10)
    ctx.destroy()
    mesh = operator.space_fe.Mesh(2, spec["cells"], spec["lo"], spec["hi"], spec["k"])
    X = mesh.node_coords()
    phi = np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])
    c = np.array(exact["c"])
    mean_ex = 1.0 * c[0] * phi                       # T(1) = 1
    var_ex = (c[1:] ** 2).sum() * phi ** 2
    se = np.sqrt(var_ex.max() / N)
    assert np.abs(mean.cpu().numpy() - mean_ex).max() <= 4 * se + 2e-3
    assert np.abs(var.cpu().numpy() - var_ex).max() <= 0.25 * var_ex.max()
    assert st["max_rel_residual"] <= 1e-10


def test_mc_errors(cuda):
    spec = I.config_small_2d_q1()
    ctx = sg.sg_setup_spec(spec)
    with pytest.raises(sg.SGError):
        sg.mc_solve_batch(ctx, np.zeros((2, 2)))        # no manufactured solution
    sg.sg_set_exact(ctx, to_product(shared_phi_exact(2, 1)))
    with pytest.raises(sg.SGError):
        sg.mc_solve_batch(ctx, np.zeros((2, 2)), batch=600)
    ctx.destroy()
