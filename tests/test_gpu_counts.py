"""Iteration counts in mesh size on the device: h-robustness of the hp-multigrid.

Theorem 3.2 makes the variable V-cycle on the lowest-order levels a preconditioner
whose condition number is bounded independently of h and eps; Section 5.2.1 reports
PCG counts that grow over the first refinements and then stay flat.  The library runs
the same iteration as the oracle (same counts in FP64, tested elsewhere), so the trend
is measured here at sizes the oracle cannot reach: the first augmented-Lagrangian
Uzawa step (FGMRES on A^eps u = F from zero, relative 1e-8) for N = 32 .. 512 with the
coarsest level 2x2, as in the paper's hierarchies.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import unit_square_hierarchy, curl_bubble_2d, forcing_at_lattice

pytestmark = pytest.mark.gpu


def _first_step_its(hdg, N, k, gamma, precision):
    nl = 1
    while 2 * 2 ** (nl - 1) < N:
        nl += 1
    ms = unit_square_hierarchy(2, nl)
    fine = ms[-1]
    fv = forcing_at_lattice(fine.coords, fine.cells, k, curl_bubble_2d().forcing(1.0, 1.0))
    ctx = hdg.hdg_setup_mesh_hierarchy(ms)
    F = hdg.hdg_condense(ctx, hdg.Params(k=k, beta=1.0, gamma=gamma, precision=precision),
                         torch.tensor(fv, device="cuda:0"))
    o = hdg.default_solve_opts()
    o.max_uzawa = 1
    _, _, info = hdg.hdg_solve(ctx, F, opts=o, raise_on_nonconvergence=False)
    ctx.close()
    return info["krylov_its"][0]


@pytest.mark.parametrize("k,gamma", [(2, 1e2), (3, 1e2)])
def test_counts_flatten_under_refinement(k, gamma):
    import paper_2303_06762_gb300 as hdg
    sizes = (32, 64, 128, 256, 512)
    its = [_first_step_its(hdg, N, k, gamma, hdg.HDG_FP64) for N in sizes]
    print(f"k={k} gamma={gamma:g}: first-step FGMRES iterations for N={sizes}: {its}")
    steps = [b - a for a, b in zip(its, its[1:])]
    # the growth per refinement dies out: at most 2 per doubling over the last two
    # doublings, and never more than the growth of the first one
    assert all(s <= 2 for s in steps[-2:]), its
    assert max(steps[1:]) <= max(steps[0], 2), its
    assert max(its) < 60, its


def test_counts_robust_in_gamma():
    """Robustness in eps: gamma = 1e4 against 1e2 on N = 32 .. 128.  (Beyond 128x128 at
    gamma = 1e4 the FP64 residual of A^eps u cannot reach the 1e-8 target, Remark 3.1:
    those first steps end stagnated, so their counts measure round-off, not the method.)"""
    import paper_2303_06762_gb300 as hdg
    sizes = (32, 64, 128)
    lo = [_first_step_its(hdg, N, 2, 1e2, hdg.HDG_FP64) for N in sizes]
    hi = [_first_step_its(hdg, N, 2, 1e4, hdg.HDG_FP64) for N in sizes]
    print(f"k=2 first-step FGMRES iterations for N={sizes}: gamma=1e2 {lo}, gamma=1e4 {hi}")
    assert all(abs(a - b) <= 3 for a, b in zip(lo, hi)), (lo, hi)


def test_lid_driven_pcg_counts_beside_the_paper():
    """The driven-lid cavity (Section 5.2.1) on hierarchies from the paper's coarsest 1/h = 2, so that
    levels 4..7 are N = 16..128: PCG counts of the first AL-Uzawa step with (nu eps)^-1 = 1e6,
    beta = 0, m = 1, variable V-cycle, printed beside Table tab:stokesLid (2D).  The meshes and the
    lid differ from the paper's (structured stand-ins, see tests/golden), so the check is the trend:
    MG_h alone within 2 of the published counts, Algorithm 2 within 8 and growing by at most 6."""
    import os
    import paper_2303_06762_gb300 as hdg
    from workloads.manufactured import dirichlet_facet_data, lid_velocity_2d
    table = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "paper_table_stokes_lid_2d.txt"))
    results = {}
    for k in (0, 1, 2, 3):
        its = []
        for nl in (4, 5, 6, 7):                       # N = 16, 32, 64, 128
            ms = unit_square_hierarchy(2, nl)
            fine = ms[-1]
            data = dirichlet_facet_data(fine.coords, fine.cells, k, lid_velocity_2d())
            zero = torch.zeros((fine.n_cells, (k + 2) * (k + 3) // 2, 2), dtype=torch.float64, device="cuda:0")
            ctx = hdg.hdg_setup_mesh_hierarchy(ms)
            F = hdg.hdg_condense(ctx, hdg.Params(k=k, nu=1.0, beta=0.0, gamma=1e6,
                                                 dirichlet=torch.tensor(data, device="cuda:0")), zero)
            o = hdg.default_solve_opts()
            o.krylov, o.max_uzawa = 1, 1
            _, _, info = hdg.hdg_solve(ctx, F, opts=o, raise_on_nonconvergence=False)
            its.append(info["krylov_its"][0])
            ctx.close()
        paper = table[table[:, 0] == k][:, 2]
        print(f"lid-driven PCG, k={k}: levels 4..7 {its}; paper (m=1, V-cycle, beta=0) {paper.astype(int).tolist()}")
        results[k] = (its, paper)
    for k, (its, paper) in results.items():
        # MG_h alone (k = 0) follows the published counts closely; Algorithm 2 (k >= 1) grows by at most
        # 6 over the four levels and stays within 8 of them
        assert np.abs(np.array(its) - paper).max() <= (2 if k == 0 else 8), (k, its, paper)
        assert max(its) - min(its) <= 6, (k, its)
