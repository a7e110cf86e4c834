"""Worker of the debug-bounds GPU test: run in a fresh process with
SG_DEBUG_BOUNDS=1, so that the binding loads libsg_debug.so (every
instrumented kernel access checked on the device).  Exercises the probe and
then the apply, multigrid, solver, Monte-Carlo and adjoint paths on small
problems; prints one JSON line with the records and a parity figure."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))


def main():
    import numpy as np
    import torch
    import paper_2605_21046_gb300 as sg
    from paper_2605_21046_gb300 import _abi
    from paper_2605_21046_gb300 import inputs as I
    from oracle import operator

    out = {"library": os.path.basename(_abi.load()._name)}
    sg.sg_debug_bounds()                                      # clear
    sg.sg_debug_bounds_probe(3, 8)
    out["probe_inside"] = sg.sg_debug_bounds()
    sg.sg_debug_bounds_probe(12, 8)
    out["probe_outside"] = sg.sg_debug_bounds()
    sg.sg_debug_bounds_probe(-1, 8)
    out["probe_negative"] = sg.sg_debug_bounds()

    # applies: FP64, double-word, transposed; 2D ragged and 3D
    specs = [dict(I.config_small_2d_q1(), cells=(13, 7)), I.scaled(I.config_3d_q2_32(), (4, 3, 5))]
    worst = 0.0
    for spec in specs:
        p = operator.SGProblem(spec)
        x = I.random_vector(spec, seed=3)
        for prec in (sg.SG_PREC_FP64, sg.SG_PREC_DW):
            ctx = sg.sg_setup_spec(spec, prec)
            for tr in (False, True):
                xd = torch.from_numpy(x).cuda()
                yd = torch.empty_like(xd)
                sg.sg_apply(ctx, 0, xd, yd, tr)
                want = p.apply(x, transpose=tr).reshape(-1)
                worst = max(worst, float(np.abs(yd.cpu().numpy() - want).max() / np.abs(want).max()))
            ctx.destroy()
    out["apply_rel_err"] = worst
    out["after_applies"] = sg.sg_debug_bounds()

    # multigrid in every precision, every level variant, and a solve
    spec = dict(I.config_small_2d_q1(), cells=(16, 16), k=2, M=3, P=2,
                coef=I.linear_sine_coef(3, 2, 0.08, [(1, 2), (2, 1), (1, 1)]))
    for prec in (sg.SG_PREC_FP64, sg.SG_PREC_FP32, sg.SG_PREC_BF16):
        ctx = sg.sg_setup_spec(spec)
        sg.sg_mg_setup(ctx, prec)
        n = ctx.info["n_unknowns"]
        r = torch.rand(n, dtype=torch.float64, device="cuda")
        z = torch.empty_like(r)
        for res in (0, 1):
            for chunk in (1, 3, 8):
                for tile in (0, 4):
                    sg.sg_mg_set_level_variant(ctx, -1, res, chunk, tile, 0)
                    sg.sg_vcycle(ctx, r, z)
                    if prec == sg.SG_PREC_BF16 and chunk <= 4:
                        sg.sg_mg_set_level_variant(ctx, -1, res, chunk, tile, 1)     # tensor-core sweep
                        sg.sg_vcycle(ctx, r, z)
        b = torch.rand(n, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        sg.sg_solve_slab(ctx, 0, b, x, rtol=1e-8)
        sg.sg_solve_slab_adjoint(ctx, 0, b, torch.zeros_like(b), rtol=1e-8)
        ctx.destroy()
    spec3 = I.scaled(I.config_3d_q2_32(), (4, 4, 4))
    ctx = sg.sg_setup_spec(spec3)
    sg.sg_mg_setup(ctx, sg.SG_PREC_BF16)
    n = ctx.info["n_unknowns"]
    sg.sg_solve_slab(ctx, 0, torch.rand(n, dtype=torch.float64, device="cuda"),
                     torch.zeros(n, dtype=torch.float64, device="cuda"), rtol=1e-8)
    ctx.destroy()
    out["after_multigrid"] = sg.sg_debug_bounds()

    # Monte-Carlo batch and the adjoint gradient
    from test_mc_gpu import shared_phi_exact
    from test_march_gpu import to_product
    spec = dict(I.config_small_2d_q1(), n_slabs=3, T=0.3)
    ctx = sg.sg_setup_spec(spec)
    sg.sg_set_exact(ctx, to_product(shared_phi_exact(2, 2)))
    xi = np.random.default_rng(4096).standard_normal((37, 2))
    sg.mc_solve_batch(ctx, xi, batch=16, mg_precision=sg.SG_PREC_FP32, rtol=1e-8)
    ctx.destroy()
    aspec = I.config_adjoint_2d(cells=(4, 4), k=2, r=1, n_slabs=3)
    ctx = sg.sg_setup_spec(aspec)
    sg.sg_set_exact(ctx, to_product(shared_phi_exact(2, 2)))
    sg.sg_mg_setup(ctx, sg.SG_PREC_FP64)
    sg.sg_adjoint_gradient(ctx, rtol=1e-10, checkpoint_every=2, cell_piece=0)
    ctx.destroy()
    out["after_mc_adjoint"] = sg.sg_debug_bounds()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
