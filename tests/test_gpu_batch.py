"""Batched solves (mg_batch_*) on the GPU.

Every member of a batch is an independent problem (its own level set, grid
size and data), so each member is held to the single-problem parity bars of
test_gpu_parity.py's mixed precision tests:
  * driven to 1e-12, within 1e-9 max|u| + 64 eps S_p of the oracle's direct
    solution (refined to fp64 exactness);
  * stopped at 1e-10, the oracle's own residual of the result is
    <= 1e-10 ||F||_inf, and the error is within 3x that of the single-problem
    fp64 V-cycle stopped at the same residual.
The batch's own behaviour: a member with NaN data (status
MG_ERR_INVALID_ARG, u = 0) and a member with zero data (u = 0, no cycles)
leave the others bit for bit as in a clean batch; graph replays, host and
device arrays and the zero-copy buffers give identical results; results do
not depend on the block size; the autotuner returns a converging choice.
The full-size case is the seeded 256-member batch (ellipses and flowers,
N in {64, 128, 256, 512}) in the launch configuration bench.py times.  The
batched fp32 V-cycle is also held to the oracle iterate by iterate (one
refinement step against the oracle's fp64 V-cycles, within the fp32 step
bound of test_gpu_mixed_parity.py) in launch shapes that select each of its
eta paths.
"""
import numpy as np
import pytest

from oracle import ghostfem as gf
from paper_2505_05105_gb300 import workloads as wl
from parity_tol import assert_solution

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_05105_gb300 import ghostmg
    ghostmg.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def small_members():
    """Members with every tail depth: N = 16..64 run wholly in shared memory,
    128 and 256 have one and two levels in global memory."""
    ps = [wl.batch_geometry(i, seed=5, sizes=(16, 32, 64, 128)) for i in range(8)]
    ps += [wl.batch_geometry(0, seed=6, sizes=(256,)), wl.flower(128, k=7, phase=0.3)]
    return ps


@pytest.fixture(scope="module")
def members():
    ps = small_members()
    sys = [gf.assemble_problem(p) for p in ps]
    Fs = [s.rhs(p.f, p.g) for p, s in zip(ps, sys)]
    ud = [gf.direct_solve(s, F) for s, F in zip(sys, Fs)]
    return ps, sys, Fs, ud


def batch(ps, **kw):
    from paper_2505_05105_gb300 import ghostmg as G
    return G.BatchSolver(ps, **kw)


def test_members_match_oracle(members):
    from paper_2505_05105_gb300 import ghostmg as G
    ps, sys, Fs, ud = members
    with batch(ps) as B:
        f, g = dev(B.pack([p.f for p in ps])), dev(B.pack([p.g for p in ps]))
        u = torch.zeros(B.total, dtype=torch.float64, device="cuda")
        info = B.solve(f, g, u, tol=1e-12)
        tight = B.unpack(host(u))
        info10 = B.solve(f, g, u, tol=1e-10)
        at10 = B.unpack(host(u))
    for k, (p, s, F, x) in enumerate(zip(ps, sys, Fs, ud)):
        assert info[k].status == G.MG_OK and info[k].rel_res <= 1e-12, (k, info[k].rel_res)
        assert info[k].n_dof == int(s.dof.sum())
        assert_solution(tight[k], x, s, F, 1e-9, what=f"member {k} N={p.N}")
        assert info10[k].status == G.MG_OK and info10[k].rel_res <= 1e-10
        r = F - s.A @ at10[k]
        assert np.abs(r[s.dof]).max() <= 1e-10 * np.abs(F).max(), k


def test_members_match_single_problem_solver(members):
    """The same member solved alone by mg_solve (mixed) and inside the batch,
    both stopped at 1e-10: the same number of fp64 checks give or take one
    (the same schedule with a different rounding order), and errors against
    the direct solution of the same order (the stopping test bounds both; a
    solve may overshoot the tolerance by a different amount, hence the
    factor and the floor of 1e-11, a tenth of the tolerance)."""
    ps, sys, Fs, ud = members
    with batch(ps) as B:
        f, g = B.pack([p.f for p in ps]), B.pack([p.g for p in ps])
        u = np.zeros(B.total)
        info = B.solve(f, g, u, tol=1e-10)
        ub = B.unpack(u)
    from paper_2505_05105_gb300 import ghostmg as G
    for k, p in enumerate(ps):
        with G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, precision="mixed") as S:
            us = torch.zeros((p.N + 1) ** 2, dtype=torch.float64, device="cuda")
            si = S.solve(dev(p.f), dev(p.g), us, tol=1e-10)
        scale = np.abs(ud[k]).max()
        e_s = np.abs(host(us) - ud[k]).max() / scale
        e_b = np.abs(ub[k] - ud[k]).max() / scale
        assert e_b <= 10 * e_s + 1e-11, (k, e_b, e_s)
        assert abs(si.checks - info[k].checks) <= 1, (k, si.checks, info[k].checks)


def test_invalid_and_zero_members_leave_the_rest_unchanged(members):
    from paper_2505_05105_gb300 import ghostmg as G
    ps = members[0][:4]
    with batch(ps) as B:
        f = B.pack([p.f for p in ps])
        g = B.pack([p.g for p in ps])
        u_clean = np.zeros(B.total)
        B.solve(f, g, u_clean, tol=1e-11)
        off = B.offsets()
        f2, g2 = f.copy(), g.copy()
        f2[off[1]:off[2]] = 0.0
        g2[off[1]:off[2]] = 0.0                   # member 1: zero data
        # member 2: NaN in g at a vertex of a cut cell, member 3: Inf in f at
        # the domain's centre (both enter F); NaN at a box corner of member 0,
        # which no cell uses, is not read
        q = ps[2]
        jc, ic = np.argwhere(gf.cell_classes(gf.snap(q.psi, q.h, 1.75)) == gf.CUT)[0]
        g2[off[2] + jc * (q.N + 1) + ic] = np.nan
        c3 = ps[3].N // 2
        f2[off[3] + c3 * (ps[3].N + 1) + c3] = np.inf
        f2[off[0]] = np.nan
        u = np.full(B.total, 5.0)
        code, info = B.solve_status(f2, g2, u, tol=1e-11)
    assert code == G.MG_ERR_INVALID_ARG
    assert [i.status for i in info] == [G.MG_OK, G.MG_OK, G.MG_ERR_INVALID_ARG,
                                        G.MG_ERR_INVALID_ARG]
    assert info[1].cycles == 0 and info[1].rel_res == 0.0
    assert np.all(u[off[1]:off[4]] == 0.0)
    np.testing.assert_array_equal(u[off[0]:off[1]], u_clean[off[0]:off[1]])


def test_replays_arrays_and_block_sizes_are_deterministic(members):
    ps = members[0]
    with batch(ps) as B:
        fh, gh = B.pack([p.f for p in ps]), B.pack([p.g for p in ps])
        a = np.zeros(B.total)
        B.solve(fh, gh, a, tol=1e-11)
        b = np.zeros(B.total)
        B.solve(fh, gh, b, tol=1e-11)                 # graph replay
        np.testing.assert_array_equal(a, b)
        ud = torch.zeros(B.total, dtype=torch.float64, device="cuda")
        B.solve(dev(fh), dev(gh), ud, tol=1e-11)      # device arrays
        np.testing.assert_array_equal(a, host(ud))
        f0, g0, u0 = B.buffers()                      # the batch's own buffers
        f0.copy_(dev(fh))
        g0.copy_(dev(gh))
        B.solve(f0, g0, u0, tol=1e-11)
        np.testing.assert_array_equal(a, host(u0))
        # pinned host arrays, read and written in place by the kernels; then
        # the own buffers again (the member table is re-pointed both times)
        fp = torch.from_numpy(fh).pin_memory()
        gp = torch.from_numpy(gh).pin_memory()
        up = torch.full((B.total,), 3.0, dtype=torch.float64).pin_memory()
        B.solve(fp, gp, up, tol=1e-11)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(a, up.numpy())
        u0.zero_()
        B.solve(f0, g0, u0, tol=1e-11)
        np.testing.assert_array_equal(a, host(u0))
        # Gauss-Seidel colour phases are free of races: neither the block
        # size nor sharing a member among the blocks of a cluster (each on
        # its own SM) changes a single bit
        for shape in ((256, 4, 1, 0), (1024, 4, 1, 0), (512, 4, 2, 0), (512, 4, 4, 0),
                      (256, 4, 8, 0), (1024, 4, 4, 20000)):
            B.set_shape(*shape)
            assert B.shape() == shape
            c = np.zeros(B.total)
            B.solve(fh, gh, c, tol=1e-11)
            np.testing.assert_array_equal(a, c)


def test_autotuner(members):
    from paper_2505_05105_gb300 import ghostmg as G
    ps, sys, Fs, ud = members
    with batch(ps) as B:
        f, g = dev(B.pack([p.f for p in ps])), dev(B.pack([p.g for p in ps]))
        (threads, first, cluster, coop), ms = B.tune(f, g, tol=1e-10, reps=2)
        assert threads in (256, 512, 1024) and first in (2, 3, 4, 6) and ms > 0.0
        assert cluster in (1, 2, 4, 8) and coop in (0, 8192, 32768, 65536, 131072)
        assert B.shape() == (threads, first, cluster, coop)
        u = torch.zeros(B.total, dtype=torch.float64, device="cuda")
        info = B.solve(f, g, u, tol=1e-10)
        _, solve_ms = B.timing()
        assert solve_ms > 0.0
        out = B.unpack(host(u))
    for k, (s, F) in enumerate(zip(sys, Fs)):
        assert info[k].status == G.MG_OK
        r = F - s.A @ out[k]
        assert np.abs(r[s.dof]).max() <= 1e-10 * np.abs(F).max()


def test_fixed_schedule():
    from paper_2505_05105_gb300 import ghostmg as G
    ps = small_members()[:3]
    with batch(ps, inner=3) as B:
        f, g = B.pack([p.f for p in ps]), B.pack([p.g for p in ps])
        info = B.solve(f, g, np.zeros(B.total), tol=1e-10)
    for i in info:
        assert i.status == G.MG_OK and i.cycles == 3 * i.checks


def test_rejects_fp64_and_bad_arguments():
    from paper_2505_05105_gb300 import ghostmg as G
    p = wl.circle64(64)
    with pytest.raises(G.GhostMGError) as e:
        s = G.mg_default_stab()
        s.precision = G.MG_FP64
        G.mg_batch_setup([G.mg_grid(p.N, p.x0, p.y0, p.h, 8)], p.psi.ravel().copy(),
                         None, s)
    assert e.value.code == G.MG_ERR_UNIMPLEMENTED
    with batch([p]) as B:
        default = B.shape()
        assert default in ((1024, 4, 2, 8192), (512, 4, 1, 0))
        with pytest.raises(G.GhostMGError) as e:
            B.solve(np.zeros(B.total), np.zeros(B.total), np.zeros(B.total), tol=-1.0)
        assert e.value.code == G.MG_ERR_INVALID_ARG
        for bad in ((384, 4, 1, 0), (512, 0, 1, 0), (512, 4, 3, 0), (512, 4, 2, -1)):
            with pytest.raises(G.GhostMGError):
                B.set_shape(*bad)
        assert B.shape() == default


def test_full_batch_256():
    """The benchmark's batch: 256 seeded members, N in {64, 128, 256, 512},
    stopped at 1e-10 in the default launch shape and with the large members
    shared by clusters of 4; sampled members (the largest of each size)
    against the oracle's direct solution."""
    from paper_2505_05105_gb300 import ghostmg as G
    ps = [wl.batch_geometry(i, seed=0) for i in range(256)]
    with batch(ps) as B:
        f, g = dev(B.pack([p.f for p in ps])), dev(B.pack([p.g for p in ps]))
        u = torch.zeros(B.total, dtype=torch.float64, device="cuda")
        info = B.solve(f, g, u, tol=1e-10)
        out = B.unpack(host(u))
        B.set_shape(512, 4, 4, 32768)
        u2 = torch.zeros_like(u)
        B.solve(f, g, u2, tol=1e-10)
        assert torch.equal(u, u2)
    assert all(i.status == G.MG_OK and i.rel_res <= 1e-10 for i in info)
    sizes = sorted({p.N for p in ps})
    assert sizes == [64, 128, 256, 512]
    for N in sizes:
        k = max((i for i, p in enumerate(ps) if p.N == N), key=lambda i: info[i].n_dof)
        s = gf.assemble_problem(ps[k])
        F = s.rhs(ps[k].f, ps[k].g)
        assert info[k].n_dof == int(s.dof.sum())
        r = F - s.A @ out[k]
        assert np.abs(r[s.dof]).max() <= 1e-10 * np.abs(F).max(), (k, N)
        if N <= 256:
            x = gf.direct_solve(s, F)
            scale = np.abs(x).max()
            # stopped at 1e-10: the error the stopping test allows, with the
            # conditioning of a Poisson problem on this grid (~ N^2)
            assert np.abs(out[k] - x).max() <= 1e-10 * N * N * scale, (k, N)


def test_batch_with_neumann_masks_and_box_sides():
    """Members with Neumann cut cells (annulus, leaf, half disc), strong box
    sides (the rectangle) and plain Dirichlet members (a flower, a seeded
    member) in one batch: each member driven to 1e-12 is within 1e-9 max|u|
    of the oracle's direct solution; NaN in one member's g_N where it enters
    F fails the call (MG_ERR_INVALID_ARG)."""
    from paper_2505_05105_gb300 import ghostmg as G
    ps = [wl.annulus(64), wl.leaf(64), wl.half_disc(64), wl.rectangle(64, 0.37),
          wl.flower(64), wl.batch_geometry(2, seed=7, sizes=(128,))]
    sys = [gf.assemble_problem(p) for p in ps]
    gNs = [p.gN if p.gN is not None else np.zeros_like(p.f) for p in ps]
    Fs = [s.rhs(p.f, p.g, gN) for p, s, gN in zip(ps, sys, gNs)]
    with batch(ps, box_sides=True) as B:
        f, g, gN = (dev(B.pack(a)) for a in ([p.f for p in ps], [p.g for p in ps], gNs))
        u = torch.zeros(B.total, dtype=torch.float64, device="cuda")
        info = B.solve(f, g, u, tol=1e-12, gN=gN)
        out = B.unpack(host(u))
        # NaN in g_N at a vertex of one of the leaf's Neumann cut cells
        q = ps[1]
        cls = gf.cell_classes(gf.snap(q.psi, q.h, 1.75))
        jc, ic = np.argwhere((cls == gf.CUT) & (np.asarray(q.neumann_mask) != 0))[0]
        bad = gN.clone()
        bad[int(B.offsets()[1]) + int(jc) * (q.N + 1) + int(ic)] = float("nan")
        with pytest.raises(G.GhostMGError) as e:
            B.solve(f, g, u, tol=1e-12, gN=bad)
        assert e.value.code == G.MG_ERR_INVALID_ARG
    for k, (p, s, F) in enumerate(zip(ps, sys, Fs)):
        assert info[k].status == G.MG_OK and info[k].rel_res <= 1e-12, (k, info[k].rel_res)
        assert info[k].n_dof == int(s.dof.sum())
        assert_solution(out[k], gf.direct_solve(s, F), s, F, 1e-9, what=p.name)



@pytest.fixture(scope="module")
def step_members():
    """Members for the step test and the oracle's V-cycles on them: the
    7-petal flower at 512^2 (4576 cut-cell vertices on its finest level: more
    eta data than one block's shared memory holds, so a team of two splits
    them), the three discs at 256^2 and the flower at 128^2 (their levels'
    eta data fit one block)."""
    from oracle import multigrid as mg
    ps = [wl.flower(512, k=7, phase=0.3), wl.three_discs(256, seed=0), wl.flower(128)]
    out = []
    for p in ps:
        s = gf.assemble_problem(p)
        lev = mg.build_hierarchy(s)
        F = s.rhs(p.f, p.g)
        refs = {}
        u = np.zeros(s.n_nodes)
        for k in (1, 2):
            u = mg.mg_cycle(lev, 0, u, F, nu1=2, nu2=1, eta=4, order="color4")
            refs[k] = u.copy()
        out.append((p, s, F, refs))
    return out


@pytest.mark.parametrize("shape", [(1024, 4, 2, 0), (1024, 4, 1, 0), (512, 4, 4, 0)],
                         ids=["pairs", "single_blocks", "clusters_of_4"])
def test_batched_step_iterates(shape, step_members):
    """The batched kernel's fp32 V-cycle held to the oracle iterate by
    iterate: a batch solve stopped after its first refinement step (a fixed
    group of `inner` fp32 V(2,1)-cycles on A e = sigma F from e = 0, then
    u = e / sigma) equals `inner` fp64 V-cycles of the oracle from u = 0
    (oracle.multigrid.mg_cycle: Sec. 4.1 smoother, Sec. 5.1 transfers, Sec.
    5.3 extra cut-cell sweeps) up to the fp32 rounding of the correction
    (parity_tol.fp32_step_tolerance, the bound of the single-problem step
    test).  The launch shapes select the eta paths: a team of two splitting
    the largest level's vertices (pairs), the lead block alone with its
    shared-memory image or window (single blocks; clusters of 4)."""
    from paper_2505_05105_gb300 import ghostmg as G
    from parity_tol import assert_nodewise, fp32_step_tolerance
    ps = [m[0] for m in step_members]
    for inner in (1, 2):
        with batch(ps, inner=inner, max_cycles=inner) as B:
            B.set_shape(*shape)
            f, g = B.pack([p.f for p in ps]), B.pack([p.g for p in ps])
            u = np.zeros(B.total)
            info = B.solve(f, g, u, tol=1e-300, allow_not_converged=True)
            out = B.unpack(u)
        for k, (p, s, F, refs) in enumerate(step_members):
            assert info[k].status == G.MG_ERR_NOT_CONVERGED and info[k].cycles == inner
            u_ref = refs[inner]
            tol, e = fp32_step_tolerance(s, F, np.zeros(s.n_nodes), u_ref, cycles=inner)
            got = out[k].ravel()
            assert_nodewise(got, u_ref, tol, (p.name, shape, inner))
            assert np.abs(got).max() >= 0.5 * np.abs(e).max()
