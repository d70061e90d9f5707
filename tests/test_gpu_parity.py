"""GPU parity: every step of the path through the C ABI against the CPU oracle.

Tolerances (from the arithmetic):
  xi             bit-exact (same correctly rounded operations on both sides)
  kappa          <= 1e-12 relative (libm vs CUDA cos/sin/exp differ by ulps;
                 the KLE sums are re-associated)
  A x            <= 1e-13 relative to |A| |x| (re-associated 9-term sums)
  per-sample Q   <= 1e-9 relative (PCG stops at rtol; the domain-mean QoI
                 error is quadratic in the energy error)
  MLMC mean      <= 1e-9 relative
"""
import numpy as np
import pytest

from oracle import fem, kle, mlmc as omlmc, philox
from synth import random_element_field, random_node_vectors, small_case, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_Q = 1e-9


@pytest.fixture(scope="module")
def m():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_11788_gb300.build import build_library
    build_library()
    import paper_2111_11788_gb300.mlmc as mod
    mod.lib()
    return mod


def stream():
    return torch.cuda.current_stream().cuda_stream


def dev(n, dtype=torch.float64):
    return torch.zeros(int(n), dtype=dtype, device="cuda")


def node_arrays_to_device(m, dim, n, arrs):
    ns = m.node_stride(dim, n)
    out = torch.zeros((arrs.shape[0], ns), dtype=torch.float64)
    out[:, :arrs.shape[1]] = torch.from_numpy(arrs)
    return out.reshape(-1).cuda()


def elem_arrays_to_device(m, dim, n, arrs):
    es = m.elem_stride(dim, n)
    out = torch.zeros((arrs.shape[0], es), dtype=torch.float64)
    out[:, :arrs.shape[1]] = torch.from_numpy(arrs)
    return out.reshape(-1).cuda()


# ---------------------------------------------------------------- A2: xi

@pytest.mark.parametrize("mpd", [1, 3, 4, 8])
def test_xi_bit_exact(m, mpd):
    M = mpd * mpd
    cfg = m.config(dim=2, n_levels=6, modes_per_dim=mpd, seed=0x0123456789ABCDEF, stream_id=7)
    with m.Plan(cfg, stream()) as plan:
        for level, first, count in ((0, 0, 37), (5, 1000, 300), (3, 2 ** 32 - 40, 40)):
            xi = dev(count * M)
            plan.draw_xi(level, first, count, xi.data_ptr())
            got = xi.cpu().numpy().reshape(count, M)
            ref = philox.draw_xi(cfg.seed, 7, level, np.arange(first, first + count), M)
            assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


def test_xi_odd_mode_count_bit_exact(m):
    # M = 9 (3 x 3): the last pair's sine branch is dropped
    cfg = m.config(dim=2, n_levels=2, modes_per_dim=3, seed=5)
    with m.Plan(cfg, stream()) as plan:
        xi = dev(33 * 9)
        plan.draw_xi(1, 0, 33, xi.data_ptr())
        ref = philox.draw_xi(5, 0, 1, np.arange(33), 9)
        assert np.array_equal(xi.cpu().numpy().reshape(33, 9).view(np.uint64), ref.view(np.uint64))


# ------------------------------------------------------------ A3/A4: kappa

@pytest.mark.parametrize("n0,levels,mpd,lam,s2", [(16, 3, 4, 0.3, 1.0), (32, 2, 8, 0.1, 1.0),
                                                  (2, 3, 5, 0.2, 2.0), (6, 2, 3, 0.25, 0.5)])
def test_kappa_parity(m, n0, levels, mpd, lam, s2):
    cfg = m.config(dim=2, n_levels=levels, coarse_cells=n0, modes_per_dim=mpd, corr_len=lam,
                   sigma2=s2, seed=1)
    M = mpd * mpd
    count = 7
    with m.Plan(cfg, stream()) as plan:
        xi = dev(count * M)
        plan.draw_xi(levels - 1, 0, count, xi.data_ptr())
        xin = xi.cpu().numpy().reshape(count, M)
        for mesh in range(levels):
            n = n0 << mesh
            es = m.elem_stride(2, n)
            kap = dev(count * es)
            plan.kappa(mesh, xi.data_ptr(), count, kap.data_ptr())
            got = kap.cpu().numpy().reshape(count, es)[:, :n * n]
            ref = kle.kappa(2, n, lam, s2, mpd, xin)
            assert np.max(np.abs(got - ref) / ref) <= 1e-12


# --------------------------------------------------------------- A5: apply

@pytest.mark.parametrize("n", [2, 5, 16, 33, 64])
def test_apply_parity(m, n):
    cfg = m.config(dim=2, n_levels=1, coarse_cells=n)
    count = 5
    x = random_node_vectors(2, n, count, seed=n)
    kap = random_element_field(2, n, count, seed=100 + n)
    with m.Plan(cfg, stream()) as plan:
        xd = node_arrays_to_device(m, 2, n, x)
        kd = elem_arrays_to_device(m, 2, n, kap)
        yd = torch.full_like(xd, np.nan)
        plan.apply(0, kd.data_ptr(), xd.data_ptr(), yd.data_ptr(), count)
        ns = m.node_stride(2, n)
        y = yd.cpu().numpy().reshape(count, ns)[:, :(n + 1) ** 2]
    for s in range(count):
        A = fem.assemble(2, n, kap[s]) if n <= 16 else fem.assemble_fast(2, n, kap[s])
        xi_ = fem.from_node_grid(2, n, x[s])
        ref = A @ xi_
        scale = abs(A) @ np.abs(xi_)
        got = fem.from_node_grid(2, n, y[s])
        assert np.all(np.abs(got - ref) <= 1e-13 * scale + 1e-300)
        full = y[s].reshape(n + 1, n + 1)
        assert np.all(full[0] == 0) and np.all(full[-1] == 0)
        assert np.all(full[:, 0] == 0) and np.all(full[:, -1] == 0)


# ----------------------------------------------------------- A6/A7: solve

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("solver,n", [("jacobi", 16), ("jacobi", 48), ("gmg", 32), ("gmg", 128),
                                      ("gmg", 4), ("jacobi", 2)])
def test_solve_parity(m, solver, n, precision):
    count = 6
    cfg = m.config(dim=2, n_levels=1, coarse_cells=n, solver=solver, rtol=1e-11,
                   precision=precision)
    kap = random_element_field(2, n, count, seed=7 * n, spread=1.0)
    with m.Plan(cfg, stream()) as plan:
        kd = elem_arrays_to_device(m, 2, n, kap)
        ns = m.node_stride(2, n)
        u = dev(count * ns)
        q = dev(count)
        it = dev(count, torch.int32)
        plan.solve(0, kd.data_ptr(), count, u.data_ptr(), q.data_ptr(), it.data_ptr())
        qh = q.cpu().numpy()
        uh = u.cpu().numpy().reshape(count, ns)[:, :(n + 1) ** 2]
        iters = it.cpu().numpy()
    assert np.all(iters > 0)
    b = fem.load_vector(2, n)
    w = fem.qoi_weights(2, n)
    for s in range(count):
        A = fem.assemble_fast(2, n, kap[s])
        uref = fem.solve_direct(A, b)
        qref = w @ uref
        assert abs(qh[s] - qref) <= RTOL_Q * abs(qref)
        assert np.max(np.abs(fem.from_node_grid(2, n, uh[s]) - uref)) <= 1e-7 * np.max(np.abs(uref))


# ------------------------------------------------- A1/A8: coupled samples

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_coupled_samples_and_level_state(m, precision):
    wl = small_case(2, n0=8, levels=3, corr_len=0.3, m=4, rtol=1e-11, precision=precision)
    cfg = m.config_from_workload(wl)
    with m.Plan(cfg, stream()) as plan:
        for level in range(3):
            qf, qc, it = plan.sample_level(level, 3, 9)
            n, mean, m2, cost = plan.level_stats(level)
            ref = [omlmc.coupled_sample(wl, level, i) for i in range(3, 12)]
            for s in range(9):
                assert abs(qf[s] - ref[s][0]) <= RTOL_Q * abs(ref[s][0])
                if level == 0:
                    assert qc[s] == 0.0
                else:
                    assert abs(qc[s] - ref[s][1]) <= RTOL_Q * abs(ref[s][1])
            st = omlmc.Welford()
            for a, b_ in ref:
                st.add(a - b_)
            assert n == 9
            assert abs(mean - st.mean) <= 1e-9 * abs(st.mean) + 1e-15
            assert abs(m2 - st.m2) <= 1e-7 * st.m2 + 1e-20
            assert cost == 9 * omlmc.level_cost(wl, level)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batching_is_bitwise_invariant(m, precision):
    """Y(l, i) and the level state do not depend on how samples are batched."""
    wl = small_case(2, n0=8, levels=3, m=4, solver="gmg", precision=precision)
    cfg = m.config_from_workload(wl)
    with m.Plan(cfg, stream()) as plan:
        qa, qca, _ = plan.sample_level(2, 0, 12)
        sa = plan.level_stats(2)
    small_ws = m.config_from_workload(wl, workspace_bytes=3 * 1024 * 1024)   # forces ragged batches
    with m.Plan(small_ws, stream()) as plan:
        q1, qc1, _ = plan.sample_level(2, 0, 5)
        q2, qc2, _ = plan.sample_level(2, 5, 7)
        sb = plan.level_stats(2)
    assert np.array_equal(qa, np.concatenate([q1, q2]))
    assert np.array_equal(qca, np.concatenate([qc1, qc2]))
    assert sa == sb


def test_empty_and_invalid_ranges(m):
    cfg = m.config(dim=2, n_levels=2, coarse_cells=4)
    with m.Plan(cfg, stream()) as plan:
        qf, qc, it = plan.sample_level(1, 0, 0)
        assert qf.size == 0
        assert plan.level_stats(1)[0] == 0
        with pytest.raises(m.MLMCError):
            plan.sample_level(2, 0, 1)
        with pytest.raises(m.MLMCError):
            plan.sample_level(0, 2 ** 32 - 1, 2)


def test_not_converged_is_reported(m):
    cfg = m.config(dim=2, n_levels=2, coarse_cells=16, max_iter=2)
    with m.Plan(cfg, stream()) as plan:
        qf, qc, it = plan.sample_level(1, 0, 3, allow_not_converged=True)
        assert np.all(it == -1)
        with pytest.raises(m.MLMCError) as e:
            plan.sample_level(1, 3, 1)
        assert e.value.status == m.MLMC_ERR_NOT_CONVERGED


# ---------------------------------------------------- A9: estimator / run

def test_allocate_matches_oracle(m):
    rng = np.random.default_rng(5)
    for _ in range(20):
        V = rng.random(6) * 10.0 ** -rng.integers(2, 9, 6)
        C = rng.random(6) * 10.0 ** rng.integers(1, 7, 6)
        eps = 10.0 ** -rng.uniform(2, 4)
        assert list(m.allocate(V, C, eps)) == omlmc.allocate(V, C, eps)


def test_fixed_n_run_config1_matches_oracle(m):
    """2D plain FP64, 16^2..64^2, Jacobi-PCG rtol 1e-11, N = (200, 50, 20)."""
    wl = workload("2d-small")
    cfg = m.config_from_workload(wl)
    N = list(wl["N"])
    with m.Plan(cfg, stream()) as plan:
        q, v, Nout = plan.run(N=N)
        states = [plan.level_stats(l) for l in range(3)]
    assert list(Nout) == N
    ref_states = []
    for l in range(3):
        st = omlmc.Welford()
        for i in range(N[l]):
            a, b_ = omlmc.coupled_sample(wl, l, i)
            st.add(a - b_)
        ref_states.append(st)
    qref, vref = omlmc.estimate(ref_states)
    assert abs(q - qref) <= RTOL_Q * abs(qref)
    assert abs(v - vref) <= 1e-6 * vref
    for (n, mean, m2, _), st in zip(states, ref_states):
        assert n == st.n and abs(mean - st.mean) <= 1e-9 * abs(st.mean) + 1e-14


def test_adaptive_run_reaches_tolerance(m):
    wl = small_case(2, n0=8, levels=3, m=4, solver="gmg", rtol=1e-10)
    cfg = m.config_from_workload(wl)
    eps = 5e-4
    with m.Plan(cfg, stream()) as plan:
        q, v, Nout = plan.run(eps=eps, pilot=10)
        states = [plan.level_stats(l) for l in range(3)]
    assert v <= eps ** 2 / 2 * (1 + 1e-9)
    V = [m2 / n for (n, _, m2, _) in states]
    C = [omlmc.level_cost(wl, l) for l in range(3)]
    need = omlmc.allocate(V, C, eps)
    assert all(int(a) >= max(10, b) for a, b in zip(Nout, need))
    # the estimate is the oracle's on exactly those samples
    ref = []
    for l in range(3):
        st = omlmc.Welford()
        for i in range(int(Nout[l])):
            a, b_ = omlmc.coupled_sample(wl, l, i)
            st.add(a - b_)
        ref.append(st)
    qref, _ = omlmc.estimate(ref)
    assert abs(q - qref) <= RTOL_Q * abs(qref)


# ------------------------------------------- graph-driven vs host-driven

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("solver", ["gmg", "jacobi"])
def test_graph_and_host_driven_solves_agree_bitwise(m, precision, solver):
    """The CUDA-graph solve (device while-loops) equals the host-driven loop bit for bit."""
    wl = small_case(2, n0=8, levels=3, m=4, solver=solver, precision=precision)
    res = []
    for graphs in (0, 1):
        cfg = m.config_from_workload(wl, use_graphs=graphs)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            with m.Plan(cfg, s.cuda_stream) as plan:
                out = [plan.sample_level(l, 0, 7) for l in range(3)]
                out.append(plan.sample_level(2, 7, 5))       # second call reuses the cached graph
                stats = [plan.level_stats(l) for l in range(3)]
                launches = plan.launch_count()
        res.append((out, stats, launches))
    (oa, sa, la), (ob, sb, lb) = res
    for (qa, ca, ia), (qb, cb, ib) in zip(oa, ob):
        assert np.array_equal(qa, qb) and np.array_equal(ca, cb) and np.array_equal(ia, ib)
    assert sa == sb
    # the graph path executes every body kernel of the converged iterations plus
    # at most one trailing no-op iteration, so its kernel count is close to the host loop's
    assert lb > 0 and la > 0 and lb < 2 * la


def test_graph_solve_on_legacy_default_stream(m):
    wl = small_case(2, n0=8, levels=2, m=4, solver="gmg")
    cfg = m.config_from_workload(wl, use_graphs=1)
    with m.Plan(cfg, 0) as plan:
        qf, qc, it = plan.sample_level(1, 0, 4)
    ref = [omlmc.coupled_sample(wl, 1, i) for i in range(4)]
    for s in range(4):
        assert abs(qf[s] - ref[s][0]) <= RTOL_Q * abs(ref[s][0])


@pytest.mark.parametrize("dim,precision", [(2, "fp64"), (2, "mixed"), (3, "fp64")])
def test_round_graph_run_matches_level_by_level(m, dim, precision):
    """mlmc_run with one graph per round (a branch per level) equals the level-by-level run bit for bit."""
    if dim == 2:
        wl = small_case(2, n0=8, levels=3, m=4, solver="gmg", precision=precision)
    else:
        wl = small_case(3, n0=4, levels=3, m=3, solver="gmg", qoi="box", precision=precision)
    out = []
    for graphs in (0, 1):
        cfg = m.config_from_workload(wl, use_graphs=graphs)
        with m.Plan(cfg, stream()) as plan:
            q, v, N = plan.run(eps=2e-3, pilot=6)
            out.append((q, v, list(N), [plan.level_stats(l) for l in range(3)], plan.launch_count()))
    assert out[0][:4] == out[1][:4]
    assert out[1][4] > 0


# ------------------------------------------------ total-order KLE truncation

@pytest.mark.parametrize("dim,n0,levels,mpd,K", [(2, 8, 3, 6, 4), (2, 5, 2, 8, 7), (3, 4, 2, 5, 3),
                                                 (3, 3, 2, 4, 0)])
def test_kappa_parity_total_order(m, dim, n0, levels, mpd, K):
    """xi has the kept-mode count; kappa = exp(Phi xi) over the kept modes (<= 1e-12)."""
    cfg = m.config(dim=dim, n_levels=levels, coarse_cells=n0, modes_per_dim=mpd, corr_len=0.2,
                   sigma2=1.4, seed=3, total_order=K)
    M = kle.n_modes(dim, mpd, K)
    assert M < mpd ** dim
    count = 5
    with m.Plan(cfg, stream()) as plan:
        xi = dev(count * M)
        plan.draw_xi(levels - 1, 2, count, xi.data_ptr())
        xin = xi.cpu().numpy().reshape(count, M)
        assert np.array_equal(xin, philox.draw_xi(3, 0, levels - 1, list(range(2, 2 + count)), M))
        for mesh in range(levels):
            n = n0 << mesh
            es = m.elem_stride(dim, n)
            kap = dev(count * es)
            plan.kappa(mesh, xi.data_ptr(), count, kap.data_ptr())
            got = kap.cpu().numpy().reshape(count, es)[:, :n ** dim]
            ref = kle.kappa(dim, n, 0.2, 1.4, mpd, xin, K)
            assert np.max(np.abs(got - ref) / ref) <= 1e-12


@pytest.mark.parametrize("dim,precision", [(2, "fp64"), (3, "mixed")])
def test_coupled_samples_total_order(m, dim, precision):
    if dim == 2:
        wl = small_case(2, n0=8, levels=2, m=6, solver="gmg", rtol=1e-11, precision=precision,
                        total_order=3)
    else:
        wl = small_case(3, n0=4, levels=2, m=4, solver="gmg", qoi="box", rtol=1e-11,
                        precision=precision, total_order=2)
    cfg = m.config_from_workload(wl)
    with m.Plan(cfg, stream()) as plan:
        qf, qc, _ = plan.sample_level(1, 0, 4)
    for s in range(4):
        rf, rc = omlmc.coupled_sample(wl, 1, s)
        assert abs(qf[s] - rf) <= RTOL_Q * abs(rf)
        assert abs(qc[s] - rc) <= RTOL_Q * abs(rc)


# ------------------------------------------------- nested initial guess

@pytest.mark.parametrize("dim,precision,solver", [(2, "fp64", "gmg"), (2, "mixed", "gmg"),
                                                  (2, "fp64", "jacobi"), (3, "fp64", "gmg"),
                                                  (3, "mixed", "gmg")])
def test_nested_guess_same_answer_fewer_iterations(m, dim, precision, solver):
    """The fine solve of a coupled sample started from the interpolated
    coarse solution meets the same stopping test: its QoIs match the oracle
    and the zero-start solve, and it needs fewer iterations on average."""
    n0, levels = (16, 3) if dim == 2 else (8, 2)
    wl = small_case(dim, n0=n0, levels=levels, corr_len=0.2, m=4, solver=solver,
                    rtol=1e-10, precision=precision)
    level = levels - 1
    out = {}
    for guess in (0, 1):
        cfg = m.config_from_workload(wl, nested_guess=guess)
        with m.Plan(cfg, stream()) as plan:
            out[guess] = plan.sample_level(level, 0, 8)
    (qf0, qc0, it0), (qf1, qc1, it1) = out[0], out[1]
    assert np.array_equal(qc0, qc1)          # the coarse solve is the same solve
    assert np.all(np.abs(qf1 - qf0) <= 2e-10 * np.abs(qf0))
    if precision == "fp64":
        assert it1.mean() < it0.mean()
    print("iterations zero start %.2f, nested guess %.2f" % (it0.mean(), it1.mean()))
    for i in (0, 5):
        rf, rc = omlmc.coupled_sample(wl, level, i)
        assert abs(qf1[i] - rf) <= RTOL_Q * abs(rf)
        assert abs(qc1[i] - rc) <= RTOL_Q * abs(rc)


def test_workspace_kept_across_plans_gives_the_same_results(m):
    """A plan that takes the workspace a destroyed plan left behind (the
    library keeps it for reuse) returns the same QoIs bit for bit, and the
    kept workspaces can be released between plans."""
    wl = small_case(2, n0=8, levels=3, m=4, solver="gmg", precision="mixed")
    cfg = m.config_from_workload(wl)
    s = torch.cuda.current_stream().cuda_stream
    got = []
    for rep in range(3):
        if rep == 2:
            m.release_cached_memory()
        with m.Plan(cfg, s) as plan:
            qf, qc, it = plan.sample_level(2, 0, 5)
        got.append((qf.tolist(), qc.tolist()))
    assert got[1] == got[0] and got[2] == got[0]
