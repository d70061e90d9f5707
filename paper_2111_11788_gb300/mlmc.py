"""ctypes binding of libmlmc (include/mlmc.h): argument marshalling only.

Every numerical step runs in the library's CUDA kernels. There is no CPU
fallback: if ``libmlmc.so`` is missing or cannot be loaded, importing the
binding raises. Device buffers are passed as raw pointers (e.g. a torch
tensor's ``data_ptr()``); streams as raw ``cudaStream_t`` handles.
"""
import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmlmc.so")

MLMC_OK = 0
MLMC_ERR_INVALID = -1
MLMC_ERR_OOM = -2
MLMC_ERR_NOT_CONVERGED = -3
MLMC_ERR_CUDA = -4
MLMC_ERR_TIMEOUT = -5
MLMC_ERR_UNIMPLEMENTED = -6

QOI_DOMAIN_MEAN = 0
QOI_BOX_MEAN = 1
JACOBI_PCG = 0
GMG_PCG = 1
FP64 = 0
MIXED = 1

# Bytes of the static device scratch of mlmc_solve_noalloc (include/mlmc.h).
NOALLOC_SCRATCH_BYTES = 64 << 20


class Config(ctypes.Structure):
    """Mirror of ``mlmc_config``."""
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("n_levels", ctypes.c_int32),
        ("coarse_cells", ctypes.c_int32),
        ("modes_per_dim", ctypes.c_int32),
        ("sigma2", ctypes.c_double),
        ("corr_len", ctypes.c_double),
        ("qoi", ctypes.c_int32),
        ("solver", ctypes.c_int32),
        ("box_lo", ctypes.c_double),
        ("box_hi", ctypes.c_double),
        ("rtol", ctypes.c_double),
        ("max_iter", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("stream_id", ctypes.c_uint32),
        ("mg_smooth", ctypes.c_int32),
        ("mg_omega", ctypes.c_double),
        ("mg_coarsest", ctypes.c_int32),
        ("check_every", ctypes.c_int32),
        ("workspace_bytes", ctypes.c_uint64),
        ("inner_rtol", ctypes.c_double),
        ("inner_max_iter", ctypes.c_int32),
        ("outer_max_iter", ctypes.c_int32),
        ("use_graphs", ctypes.c_int32),
        ("total_order", ctypes.c_int32),
        ("z_chunk", ctypes.c_int32),
        ("nested_guess", ctypes.c_int32),
        ("kle_tensor", ctypes.c_int32),
        ("stencil_tile", ctypes.c_int32),
        ("batch_split", ctypes.c_int32),
    ]


class LevelState(ctypes.Structure):
    """Mirror of ``mlmc_level_state``."""
    _fields_ = [("n", ctypes.c_int64), ("mean", ctypes.c_double), ("m2", ctypes.c_double),
                ("cost_sum", ctypes.c_double)]


class KernelStat(ctypes.Structure):
    """Mirror of ``mlmc_kernel_stat``."""
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    """Mirror of ``mlmc_server_config``."""
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("max_slots", ctypes.c_int32),
                ("pilot", ctypes.c_int32), ("device", ctypes.c_int32),
                ("max_rounds", ctypes.c_int32), ("adapt_from", ctypes.c_int32),
                ("solo_rounds", ctypes.c_int32)]


class RequestResult(ctypes.Structure):
    """Mirror of ``mlmc_request_result``."""
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("group_rounds", ctypes.c_int32),
                ("q_hat", ctypes.c_double), ("stat_var", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("dof_solves", ctypes.c_double),
                ("N", ctypes.c_int64 * 16)]


class TuneReport(ctypes.Structure):
    """Mirror of ``mlmc_tune_report``."""
    _fields_ = [("candidates", ctypes.c_int32), ("z_chunk", ctypes.c_int32),
                ("inner_rtol", ctypes.c_double), ("mg_omega", ctypes.c_double),
                ("best_ms", ctypes.c_double), ("worst_ms", ctypes.c_double),
                ("stencil_tile", ctypes.c_int32), ("batch_split", ctypes.c_int32)]


TUNE_INNER_RTOL = 1
TUNE_MG_OMEGA = 2
TUNE_Z_CHUNK = 4
TUNE_TILE = 8
TUNE_BATCH = 16


class SchedResult(ctypes.Structure):
    """Mirror of ``mlmc_sched_result``."""
    _fields_ = [("makespan", ctypes.c_double), ("work_total", ctypes.c_double),
                ("work_lb", ctypes.c_double), ("last_start", ctypes.c_double),
                ("idle_before_last", ctypes.c_double), ("batches", ctypes.c_int64)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)
_I32P = ctypes.POINTER(ctypes.c_int32)
_I64P = ctypes.POINTER(ctypes.c_int64)

# (name, restype, argtypes) for every symbol of include/mlmc.h and include/mlmc_server.h
SIGNATURES = [
    ("mlmc_config_default", None, [ctypes.POINTER(Config)]),
    ("mlmc_node_stride", _I64, [_I, _I]),
    ("mlmc_elem_stride", _I64, [_I, _I]),
    ("mlmc_mesh_cells", _I64, [ctypes.POINTER(Config), _I]),
    ("mlmc_level_cost", _D, [ctypes.POINTER(Config), _I]),
    ("mlmc_coef_count", _I64, [ctypes.POINTER(Config)]),
    ("mlmc_status_str", ctypes.c_char_p, [_I]),
    ("mlmc_plan_create", _I, [ctypes.POINTER(Config), _P, ctypes.POINTER(_P)]),
    ("mlmc_plan_destroy", _I, [_P]),
    ("mlmc_release_cached_memory", _I, []),
    ("mlmc_reset_stats", _I, [_P]),
    ("mlmc_sample_level", _I, [_P, _I, _I64, _I64, _DP, _DP, _I32P]),
    ("mlmc_level_stats", _I, [_P, _I, ctypes.POINTER(LevelState)]),
    ("mlmc_estimate", _I, [_P, _DP, _DP]),
    ("mlmc_allocate", _I, [_DP, _DP, _I, _D, _I64P]),
    ("mlmc_run", _I, [_P, _D, _I64, _I64P, _DP, _DP, _I64P]),
    ("mlmc_draw_xi", _I, [_P, _I, _I64, _I64, _P]),
    ("mlmc_kappa", _I, [_P, _I, _P, _I64, _P]),
    ("mlmc_kappa32", _I, [_P, _I, _P, _I64, _P]),
    ("mlmc_apply", _I, [_P, _I, _P, _P, _P, _I64]),
    ("mlmc_apply32", _I, [_P, _I, _P, _P, _P, _I64]),
    ("mlmc_solve", _I, [_P, _I, _P, _I64, _P, _P, _P]),
    ("mlmc_kernel_count", _I, []),
    ("mlmc_kernel_name", ctypes.c_char_p, [_I]),
    ("mlmc_profile_enable", _I, [_P, _I]),
    ("mlmc_profile_reset", _I, [_P]),
    ("mlmc_kernel_stats", _I, [_P, _I, ctypes.POINTER(KernelStat)]),
    ("mlmc_launch_count", _I64, [_P]),
    ("mlmc_solve_noalloc", _I, [ctypes.POINTER(Config), _I, _P, _I64, _P, _P, _P]),
    ("mlmc_round_begin", _I, [_P, _I64P, _I64P]),
    ("mlmc_round_ready", _I, [_P]),
    ("mlmc_round_end", _I, [_P]),
    ("mlmc_allocation", _I, [_P, _D, _I64P]),
    ("mlmc_round_values", _I, [_P, _I, _DP, _DP, _I64]),
    ("mlmc_round_begin_group", _I, [ctypes.POINTER(_P), _I, _I64P, _I64P, _P, ctypes.c_uint64]),
    ("mlmc_round_bytes_group", _I64, [ctypes.POINTER(ctypes.POINTER(Config)), _I, _I64P]),
    ("mlmc_round_end_group", _I, [_P, _I32P]),
    ("mlmc_plan_retarget", _I, [_P, ctypes.POINTER(Config)]),
    ("mlmc_round_bytes", _I64, [ctypes.POINTER(Config), _I64P]),
    ("mlmc_plan_set_workspace", _I, [_P, _P, ctypes.c_uint64]),
    ("mlmc_run_adaptive", _I, [_P, _D, _I64, ctypes.c_int32, _DP, _DP, _I64P, _I32P]),
    ("mlmc_level_fold", _I, [_P, _I, _DP, _DP, _I64]),
    ("mlmc_autotune", _I, [_P, _I, _I64, _I, ctypes.POINTER(TuneReport)]),
    ("mlmc_probe_fp64_rate", _I, [_P, _DP, _DP]),
    # include/mlmc_sched.h
    ("mlmc_batch_size", _I64, [_I64, _I64, _I64, _D, _D]),
    ("mlmc_schedule_greedy", _I, [_I, _I64P, _I64P, _DP, _I64, _I, _D, _D, _D,
                                  ctypes.POINTER(SchedResult), _DP]),
    ("mlmc_adapt", _I, [_P, ctypes.c_int32, _D, _I64P, _I32P, _DP]),
    # include/mlmc_server.h
    ("mlmc_server_create", _I, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)]),
    ("mlmc_server_submit", _I, [_P, ctypes.POINTER(Config), _D, ctypes.POINTER(ctypes.c_uint64)]),
    ("mlmc_server_poll", _I, [_P, ctypes.c_uint64, ctypes.POINTER(_I), ctypes.POINTER(RequestResult)]),
    ("mlmc_server_drain", _I, [_P, _D]),
    ("mlmc_server_clock", _D, [_P]),
    ("mlmc_server_destroy", _I, [_P]),
]


def load(path=LIB_PATH):
    """Load libmlmc.so and declare every entry point. Raises if it is missing."""
    if not os.path.exists(path):
        raise ImportError("libmlmc.so not built (run __graft_entry__.build()): " + path)
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


class MLMCError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        msg = lib().mlmc_status_str(status).decode()
        super().__init__("%s: %s (%d)" % (what, msg, status))


def check(status, what, allow=()):
    if status != MLMC_OK and status not in allow:
        raise MLMCError(status, what)
    return status


def _dp(arr):
    return None if arr is None else arr.ctypes.data_as(_DP)


def config(dim=2, n_levels=3, coarse_cells=16, modes_per_dim=4, sigma2=1.0, corr_len=0.3,
           qoi="domain", solver="jacobi", box=(0.25, 0.75), rtol=1e-10, max_iter=None,
           precision="fp64", seed=0, stream_id=0, mg_omega=None, check_every=0,
           workspace_bytes=0, inner_rtol=None, inner_max_iter=None, outer_max_iter=None,
           use_graphs=None, total_order=None, nested_guess=None, kle_tensor=None,
           stencil_tile=None, batch_split=None):
    """Build a Config from plain values (defaults from mlmc_config_default)."""
    c = Config()
    lib().mlmc_config_default(ctypes.byref(c))
    c.dim, c.n_levels, c.coarse_cells, c.modes_per_dim = dim, n_levels, coarse_cells, modes_per_dim
    c.sigma2, c.corr_len = sigma2, corr_len
    c.qoi = {"domain": QOI_DOMAIN_MEAN, "box": QOI_BOX_MEAN}[qoi]
    c.solver = {"jacobi": JACOBI_PCG, "gmg": GMG_PCG}[solver]
    c.box_lo, c.box_hi = box
    c.rtol = rtol
    if max_iter is not None:
        c.max_iter = max_iter
    elif solver == "gmg":
        c.max_iter = 500
    c.precision = {"fp64": FP64, "mixed": MIXED}[precision]
    c.seed, c.stream_id = seed, stream_id
    if mg_omega is not None:
        c.mg_omega = mg_omega
    c.check_every = check_every
    c.workspace_bytes = workspace_bytes
    if inner_rtol is not None:
        c.inner_rtol = inner_rtol
    if inner_max_iter is not None:
        c.inner_max_iter = inner_max_iter
    if outer_max_iter is not None:
        c.outer_max_iter = outer_max_iter
    if use_graphs is not None:
        c.use_graphs = int(use_graphs)
    if total_order is not None:
        c.total_order = int(total_order)
    if nested_guess is not None:
        c.nested_guess = int(nested_guess)
    if kle_tensor is not None:
        c.kle_tensor = int(kle_tensor)
    if stencil_tile is not None:
        c.stencil_tile = int(stencil_tile)
    if batch_split is not None:
        c.batch_split = int(batch_split)
    return c


def config_from_workload(wl, **over):
    """Config from a workload dictionary (see synth.workloads)."""
    args = dict(dim=wl["dim"], n_levels=wl["levels"], coarse_cells=wl["n0"],
                modes_per_dim=wl["m"], sigma2=wl["sigma2"], corr_len=wl["corr_len"],
                qoi=wl.get("qoi", "domain"), solver=wl.get("solver", "jacobi"),
                box=tuple(wl.get("box", (0.25, 0.75))), rtol=wl["rtol"],
                seed=wl.get("seed", 0), stream_id=wl.get("stream_id", 0),
                precision=wl.get("precision", "fp64"),
                total_order=-1 if wl.get("total_order") is None else wl["total_order"])
    args.update(over)
    return config(**args)


def probe_fp64_rate(stream=0):
    """Measured FP64 FMA rate of the current device: (TFLOP/s, best launch ms)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    check(lib().mlmc_probe_fp64_rate(_P(stream), ctypes.byref(tf), ctypes.byref(ms)),
          "mlmc_probe_fp64_rate")
    return tf.value, ms.value


def round_bytes_group(cfgs, count):
    """mlmc_round_bytes_group for configurations cfgs and counts (len(cfgs) x n_levels)."""
    import numpy as np
    arr = (ctypes.POINTER(Config) * len(cfgs))(*[ctypes.pointer(c) for c in cfgs])
    c = np.ascontiguousarray(count, dtype=np.int64).reshape(-1)
    return int(lib().mlmc_round_bytes_group(arr, len(cfgs), c.ctypes.data_as(_I64P)))


def round_group(plans, first, count, ws_ptr, ws_bytes):
    """mlmc_round_begin_group + mlmc_round_end_group on plans[0]: returns
    (status, per-plan flags of solves that hit their iteration cap)."""
    import numpy as np
    hs = (_P * len(plans))(*[p._h for p in plans])
    f = np.ascontiguousarray(first, dtype=np.int64).reshape(-1)
    c = np.ascontiguousarray(count, dtype=np.int64).reshape(-1)
    check(lib().mlmc_round_begin_group(hs, len(plans), f.ctypes.data_as(_I64P), c.ctypes.data_as(_I64P),
                                       _P(ws_ptr), ctypes.c_uint64(ws_bytes)), "mlmc_round_begin_group")
    bad = np.zeros(len(plans), dtype=np.int32)
    st = lib().mlmc_round_end_group(plans[0]._h, bad.ctypes.data_as(_I32P))
    if st not in (MLMC_OK, MLMC_ERR_NOT_CONVERGED):
        check(st, "mlmc_round_end_group")
    return st, bad


def release_cached_memory():
    """mlmc_release_cached_memory: workspaces kept from destroyed plans back to the driver."""
    check(lib().mlmc_release_cached_memory(), "mlmc_release_cached_memory")


def coef_count(cfg):
    """mlmc_coef_count: KLE coefficients per sample of a configuration."""
    return int(lib().mlmc_coef_count(ctypes.byref(cfg)))


def node_stride(dim, n):
    return lib().mlmc_node_stride(dim, n)


def elem_stride(dim, n):
    return lib().mlmc_elem_stride(dim, n)


class Plan:
    """An mlmc_plan: KLE tables, level states and workspace on one device."""

    def __init__(self, cfg, stream=0):
        self.cfg = cfg
        self._h = _P()
        check(lib().mlmc_plan_create(ctypes.byref(cfg), _P(stream), ctypes.byref(self._h)),
              "mlmc_plan_create")

    def close(self):
        if self._h:
            check(lib().mlmc_plan_destroy(self._h), "mlmc_plan_destroy")
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- plan-level API (host outputs) ---
    def mesh_cells(self, mesh):
        return lib().mlmc_mesh_cells(ctypes.byref(self.cfg), mesh)

    def sample_level(self, level, first, count, want=True, allow_not_converged=False):
        import numpy as np
        qf = np.zeros(count) if want else None
        qc = np.zeros(count) if want else None
        it = np.zeros(count, dtype=np.int32) if want else None
        st = lib().mlmc_sample_level(self._h, level, first, count, _dp(qf), _dp(qc),
                                     None if it is None else it.ctypes.data_as(_I32P))
        check(st, "mlmc_sample_level",
              allow=(MLMC_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return qf, qc, it

    def level_stats(self, level):
        s = LevelState()
        check(lib().mlmc_level_stats(self._h, level, ctypes.byref(s)), "mlmc_level_stats")
        return s.n, s.mean, s.m2, s.cost_sum

    def estimate(self):
        q, v = ctypes.c_double(), ctypes.c_double()
        check(lib().mlmc_estimate(self._h, ctypes.byref(q), ctypes.byref(v)), "mlmc_estimate")
        return q.value, v.value

    def reset_stats(self):
        check(lib().mlmc_reset_stats(self._h), "mlmc_reset_stats")

    def run(self, eps=None, pilot=0, N=None):
        import numpy as np
        L1 = self.cfg.n_levels
        q, v = ctypes.c_double(), ctypes.c_double()
        Nout = np.zeros(L1, dtype=np.int64)
        Nfix = None if N is None else np.ascontiguousarray(N, dtype=np.int64)
        st = lib().mlmc_run(self._h, eps or 0.0, pilot,
                            None if Nfix is None else Nfix.ctypes.data_as(_I64P),
                            ctypes.byref(q), ctypes.byref(v), Nout.ctypes.data_as(_I64P))
        check(st, "mlmc_run")
        return q.value, v.value, Nout

    def autotune(self, level, count, flags=31):
        """mlmc_autotune: keep the fastest setting; returns the report as a dict."""
        r = TuneReport()
        check(lib().mlmc_autotune(self._h, int(level), int(count), int(flags), ctypes.byref(r)),
              "mlmc_autotune")
        return dict(candidates=r.candidates, z_chunk=r.z_chunk, inner_rtol=r.inner_rtol,
                    mg_omega=r.mg_omega, stencil_tile=r.stencil_tile, batch_split=r.batch_split,
                    best_ms=r.best_ms, worst_ms=r.worst_ms)

    def allocation(self, eps):
        """mlmc_allocation: N_l of Eq. (mlmc_num_samples) from the device level states."""
        import numpy as np
        N = np.zeros(self.cfg.n_levels, dtype=np.int64)
        check(lib().mlmc_allocation(self._h, float(eps), N.ctypes.data_as(_I64P)), "mlmc_allocation")
        return N

    def round(self, first, count):
        """mlmc_round_begin + mlmc_round_end: samples first[l] .. first[l] + count[l] - 1
        of every level as one graph-captured round; folded into the level states."""
        import numpy as np
        f = np.ascontiguousarray(first, dtype=np.int64)
        c = np.ascontiguousarray(count, dtype=np.int64)
        check(lib().mlmc_round_begin(self._h, f.ctypes.data_as(_I64P), c.ctypes.data_as(_I64P)),
              "mlmc_round_begin")
        check(lib().mlmc_round_end(self._h), "mlmc_round_end")

    def round_begin(self, first, count):
        """mlmc_round_begin (asynchronous); see round_ready / round_end."""
        import numpy as np
        f = np.ascontiguousarray(first, dtype=np.int64)
        c = np.ascontiguousarray(count, dtype=np.int64)
        check(lib().mlmc_round_begin(self._h, f.ctypes.data_as(_I64P), c.ctypes.data_as(_I64P)),
              "mlmc_round_begin")

    def round_ready(self):
        return lib().mlmc_round_ready(self._h)

    def round_end(self):
        return lib().mlmc_round_end(self._h)

    def round_values(self, level, count):
        """mlmc_round_values: (Q_l, Q_{l-1}) of the last finished round's samples of `level`."""
        import numpy as np
        qf = np.zeros(count, dtype=np.float64)
        qc = np.zeros(count, dtype=np.float64)
        check(lib().mlmc_round_values(self._h, int(level), _dp(qf), _dp(qc), int(count)),
              "mlmc_round_values")
        return qf, qc

    def level_fold(self, level, qf, qc=None):
        """mlmc_level_fold: fold host sample values into the level state, in order."""
        import numpy as np
        qf = np.ascontiguousarray(qf, dtype=np.float64)
        qc = None if qc is None else np.ascontiguousarray(qc, dtype=np.float64)
        check(lib().mlmc_level_fold(self._h, int(level), _dp(qf), _dp(qc), int(qf.size)),
              "mlmc_level_fold")

    def run_adaptive(self, eps, pilot, L0):
        """mlmc_run_adaptive: returns (q_hat, stat_var, N per level, final level)."""
        import numpy as np
        q, v = ctypes.c_double(), ctypes.c_double()
        Nout = np.zeros(self.cfg.n_levels, dtype=np.int64)
        L = ctypes.c_int32()
        check(lib().mlmc_run_adaptive(self._h, float(eps), int(pilot), int(L0), ctypes.byref(q),
                                      ctypes.byref(v), Nout.ctypes.data_as(_I64P), ctypes.byref(L)),
              "mlmc_run_adaptive")
        return q.value, v.value, Nout, L.value

    def adapt(self, L_active, eps):
        """mlmc_adapt: (N for levels 0..L_active, new level, (alpha, c))."""
        import numpy as np
        N = np.zeros(L_active + 1, dtype=np.int64)
        L = ctypes.c_int32()
        fit = (ctypes.c_double * 2)()
        check(lib().mlmc_adapt(self._h, int(L_active), float(eps), N.ctypes.data_as(_I64P),
                               ctypes.byref(L), fit), "mlmc_adapt")
        return N, L.value, (fit[0], fit[1])

    # --- device-level API (raw device pointers) ---
    def draw_xi(self, level, first, count, xi_ptr):
        check(lib().mlmc_draw_xi(self._h, level, first, count, _P(xi_ptr)), "mlmc_draw_xi")

    def kappa(self, mesh, xi_ptr, count, kappa_ptr):
        check(lib().mlmc_kappa(self._h, mesh, _P(xi_ptr), count, _P(kappa_ptr)), "mlmc_kappa")

    def kappa32(self, mesh, xi_ptr, count, kappa32_ptr):
        check(lib().mlmc_kappa32(self._h, mesh, _P(xi_ptr), count, _P(kappa32_ptr)), "mlmc_kappa32")

    def apply(self, mesh, kappa_ptr, x_ptr, y_ptr, count):
        check(lib().mlmc_apply(self._h, mesh, _P(kappa_ptr), _P(x_ptr), _P(y_ptr), count),
              "mlmc_apply")

    def apply32(self, mesh, kappa32_ptr, x_ptr, y_ptr, count):
        check(lib().mlmc_apply32(self._h, mesh, _P(kappa32_ptr), _P(x_ptr), _P(y_ptr), count),
              "mlmc_apply32")

    def solve(self, mesh, kappa_ptr, count, u_ptr, q_ptr, iters_ptr, allow_not_converged=False):
        st = lib().mlmc_solve(self._h, mesh, _P(kappa_ptr), count, _P(u_ptr or None),
                              _P(q_ptr), _P(iters_ptr or None))
        return check(st, "mlmc_solve",
                     allow=(MLMC_ERR_NOT_CONVERGED,) if allow_not_converged else ())

    # --- tracing ---
    def profile(self, mask=-1):
        """Trace kernels selected by bit mask (1 << kernel id; -1 all, 0 off)."""
        check(lib().mlmc_profile_enable(self._h, int(mask)), "mlmc_profile_enable")

    def profile_reset(self):
        check(lib().mlmc_profile_reset(self._h), "mlmc_profile_reset")

    def kernel_stats(self):
        out = {}
        for k in range(lib().mlmc_kernel_count()):
            s = KernelStat()
            check(lib().mlmc_kernel_stats(self._h, k, ctypes.byref(s)), "mlmc_kernel_stats")
            out[lib().mlmc_kernel_name(k).decode()] = (s.launches, s.ms, s.bytes)
        return out

    @staticmethod
    def kernel_id(name):
        for k in range(lib().mlmc_kernel_count()):
            if lib().mlmc_kernel_name(k).decode() == name:
                return k
        raise KeyError(name)

    def launch_count(self):
        return lib().mlmc_launch_count(self._h)


class Server:
    """An mlmc_server: continuous-batching MLMC estimation requests.

    ``submit(cfg, eps)`` queues one adaptive estimation and returns its id;
    ``poll(id)`` returns None while it runs, else a dict of its result
    (times in seconds on the server clock)."""

    def __init__(self, hbm_budget=0, max_slots=8, pilot=32, device=0, max_rounds=0, adapt_from=0,
                 solo_rounds=0):
        sc = ServerConfig(hbm_budget=int(hbm_budget), max_slots=int(max_slots), pilot=int(pilot),
                          device=int(device), max_rounds=int(max_rounds),
                          adapt_from=int(adapt_from), solo_rounds=int(solo_rounds))
        self._h = _P()
        check(lib().mlmc_server_create(ctypes.byref(sc), ctypes.byref(self._h)),
              "mlmc_server_create")

    def submit(self, cfg, eps):
        rid = ctypes.c_uint64()
        check(lib().mlmc_server_submit(self._h, ctypes.byref(cfg), float(eps), ctypes.byref(rid)),
              "mlmc_server_submit")
        return rid.value

    def poll(self, rid):
        done = ctypes.c_int()
        r = RequestResult()
        check(lib().mlmc_server_poll(self._h, rid, ctypes.byref(done), ctypes.byref(r)),
              "mlmc_server_poll")
        if not done.value:
            return None
        n = [int(x) for x in r.N]
        return dict(id=r.id, status=r.status, rounds=r.rounds, levels=r.levels,
                    group_rounds=r.group_rounds, q_hat=r.q_hat,
                    stat_var=r.stat_var, t_submit=r.t_submit, t_admit=r.t_admit,
                    t_done=r.t_done, dof_solves=r.dof_solves, N=n)

    def drain(self, timeout=600.0):
        check(lib().mlmc_server_drain(self._h, float(timeout)), "mlmc_server_drain")

    def clock(self):
        return lib().mlmc_server_clock(self._h)

    def close(self):
        if self._h:
            check(lib().mlmc_server_destroy(self._h), "mlmc_server_destroy")
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def batch_size(N, n, parts, min_frac=0.01, max_frac=0.6180339887498949):
    """mlmc_batch_size: the next batch of a level by Eq. (batch) (-1: invalid)."""
    return lib().mlmc_batch_size(int(N), int(n), int(parts), float(min_frac), float(max_frac))


def schedule_greedy(q, n_tasks, w, p, batch=False, min_frac=0.01, max_frac=0.6180339887498949,
                    dispatch_cost=0.0, want_starts=False):
    """mlmc_schedule_greedy: simulate Algorithm 1; returns (result dict, starts or None)."""
    import numpy as np
    L = len(q)
    qa = np.ascontiguousarray(q, dtype=np.int64)
    na = np.ascontiguousarray(n_tasks, dtype=np.int64)
    wa = np.ascontiguousarray(w, dtype=np.float64)
    st = np.zeros(wa.size) if want_starts else None
    r = SchedResult()
    check(lib().mlmc_schedule_greedy(L, qa.ctypes.data_as(_I64P), na.ctypes.data_as(_I64P),
                                     _dp(wa), int(p), int(bool(batch)), float(min_frac),
                                     float(max_frac), float(dispatch_cost), ctypes.byref(r),
                                     _dp(st)), "mlmc_schedule_greedy")
    return (dict(makespan=r.makespan, work_total=r.work_total, work_lb=r.work_lb,
                 last_start=r.last_start, idle_before_last=r.idle_before_last,
                 batches=r.batches), st)


def allocate(V, C, eps):
    """Eq. (mlmc_num_samples) evaluated by the library (on the device)."""
    import numpy as np
    V = np.ascontiguousarray(V, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.float64)
    N = np.zeros(V.size, dtype=np.int64)
    check(lib().mlmc_allocate(_dp(V), _dp(C), V.size, eps, N.ctypes.data_as(_I64P)),
          "mlmc_allocate")
    return N
