"""Python binding of libclr.so (ctypes).  Argument marshalling only: every step
of the solver runs in the library.  Function names follow include/clr.h.

The library is built in-tree by ``paper_2412_19027_gb300.build.build()``; if
it is missing every call raises ``RuntimeError`` (there is no fallback)."""
import ctypes as C
import os

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libclr.so")

STATUS = {0: "UNSOLVED", 1: "SOLVED", 2: "PRIMAL_INFEASIBLE", 3: "DUAL_INFEASIBLE", 4: "MAX_ITER",
          5: "INSUFFICIENT_PROGRESS", 6: "NUMERICAL_ERROR"}


class ClrError(RuntimeError):
    def __init__(self, code, where):
        msg = "%s failed: %s (%d)" % (where, _err_string(code), code)
        if code == -5:
            msg += ": " + _lib().clr_last_cuda_error().decode()
        super().__init__(msg)
        self.code = code


class clr_cone(C.Structure):
    _fields_ = [("type", C.c_int32), ("dim", C.c_int32), ("alpha", C.c_double)]


class clr_csc(C.Structure):
    _fields_ = [("nrows", C.c_int64), ("ncols", C.c_int64), ("nnz", C.c_int64), ("colptr", C.POINTER(C.c_int64)),
                ("rowind", C.POINTER(C.c_int32)), ("val", C.POINTER(C.c_double))]


class clr_settings(C.Structure):
    _fields_ = [("eps_feas", C.c_double), ("eps_inf", C.c_double), ("max_iter", C.c_int32),
                ("factor_bits", C.c_int32), ("static_reg", C.c_double), ("static_reg_dyn", C.c_double),
                ("dyn_reg_eps", C.c_double), ("dyn_reg_delta", C.c_double), ("ir_max_steps", C.c_int32),
                ("ir_abstol", C.c_double), ("ir_reltol", C.c_double), ("ir_stop_ratio", C.c_double),
                ("equilibrate", C.c_int32),
                ("ruiz_passes", C.c_int32), ("scale_min", C.c_double), ("scale_max", C.c_double),
                ("step_fraction", C.c_double), ("backtrack", C.c_double), ("nbhd_beta", C.c_double),
                ("min_step", C.c_double), ("use_graph", C.c_int32), ("verbose", C.c_int32),
                ("fp64_escalation", C.c_int32), ("big_front_schedule", C.c_int32),
                ("small_front_max", C.c_int32), ("amalgamation", C.c_int32), ("escalate_ratio", C.c_double),
                ("soc_expand_dim", C.c_int32), ("pull_lists_direct", C.c_int32)]


class clr_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("ir_steps_total", C.c_int32),
                ("dyn_reg_hits", C.c_int32), ("obj_primal", C.c_double), ("obj_dual", C.c_double),
                ("res_primal", C.c_double), ("res_dual", C.c_double), ("gap_abs", C.c_double),
                ("gap_rel", C.c_double), ("mu", C.c_double), ("tau", C.c_double), ("kappa", C.c_double),
                ("setup_s", C.c_double), ("solve_s", C.c_double), ("fp64_from_iter", C.c_int32),
                ("pad", C.c_int32)]


class clr_cone_times(C.Structure):
    _fields_ = [("scaling_ms", C.c_double), ("step_ms", C.c_double), ("combined_ds_ms", C.c_double),
                ("rows", C.c_int64), ("kkt_values", C.c_int64)]


class clr_tune_result(C.Structure):
    _fields_ = [("small_front_max", C.c_int32), ("amalgamation", C.c_int32), ("big_front_schedule", C.c_int32),
                ("candidates", C.c_int32), ("ms_per_iter", C.c_double), ("base_ms_per_iter", C.c_double),
                ("from_cache", C.c_int32), ("pad", C.c_int32)]


class clr_symbolic_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("kkt_dim", C.c_int64), ("kkt_nnz_lower", C.c_int64),
                ("l_nnz", C.c_int64), ("factor_flops", C.c_double), ("n_supernodes", C.c_int64),
                ("n_levels", C.c_int64), ("max_front", C.c_int64), ("front_pool_entries", C.c_int64),
                ("n_dense_rows", C.c_int64), ("ordering", C.c_int64), ("l_nnz_exact", C.c_int64),
                ("l_nnz_counted", C.c_int64), ("factor_flops_stored", C.c_double), ("maps_digest", C.c_uint64)]


class clr_problem(C.Structure):
    _fields_ = [("P_upper", C.POINTER(clr_csc)), ("q", C.POINTER(C.c_double)), ("A", C.POINTER(clr_csc)),
                ("b", C.POINTER(C.c_double)), ("cones", C.POINTER(clr_cone)), ("ncones", C.c_int32)]


class clr_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("cohorts", C.c_int64), ("max_cohort_seen", C.c_int64), ("peak_bytes", C.c_int64),
                ("bytes_in_use", C.c_int64)]


class clr_perf(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("iterations", C.c_int32), ("factorizations", C.c_int32),
                ("init_ms", C.c_double), ("resid_cones_ms", C.c_double), ("factor_ms", C.c_double),
                ("solve_step_ms", C.c_double), ("factor_flops", C.c_double), ("factor64_ms", C.c_double),
                ("factorizations64", C.c_int32), ("pad", C.c_int32)]


_LIB = None
EXPORTS = ["clr_default_settings", "clr_setup", "clr_analyze", "clr_solve", "clr_get_solution", "clr_update_qb",
           "clr_update_PA", "clr_batch_update_PA",
           "clr_get_symbolic_stats", "clr_get_perf", "clr_get_symbolic", "clr_get_scaling", "clr_get_history", "clr_set_stream",
           "clr_set_allocator", "clr_free", "clr_error_string", "clr_status_string", "clr_last_cuda_error",
           "clr_cones_scaling", "clr_cones_step_length", "clr_cones_combined_ds", "clr_cones_time", "clr_ldl_solve",
           "clr_dense_ldl_solve_noalloc", "clr_batch_setup", "clr_batch_analyze", "clr_batch_size", "clr_batch_get",
           "clr_batch_update_qb", "clr_server_create", "clr_server_submit", "clr_server_poll", "clr_server_wait",
           "clr_server_get_stats", "clr_server_destroy", "clr_autotune", "clr_probe_peaks", "clr_solve_begin",
           "clr_solve_iterate", "clr_solve_end"]


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libclr.so is not built; run paper_2412_19027_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER
        vp = C.c_void_p
        L.clr_default_settings.argtypes = [P(clr_settings), C.c_int32]
        for name in ("clr_setup", "clr_analyze"):
            getattr(L, name).argtypes = [P(vp), P(clr_csc), P(C.c_double), P(clr_csc), P(C.c_double), P(clr_cone),
                                         C.c_int32, P(clr_settings)]
        L.clr_solve.argtypes = [vp]
        L.clr_get_solution.argtypes = [vp, P(C.c_double), P(C.c_double), P(C.c_double), P(clr_info)]
        L.clr_update_qb.argtypes = [vp, P(C.c_double), P(C.c_double)]
        L.clr_update_PA.argtypes = [vp, P(C.c_double), P(C.c_double)]
        L.clr_batch_update_PA.argtypes = [vp, C.c_int32, P(C.c_double), P(C.c_double)]
        L.clr_get_symbolic_stats.argtypes = [vp, P(clr_symbolic_stats)]
        L.clr_get_perf.argtypes = [vp, P(clr_perf)]
        L.clr_get_symbolic.argtypes = [vp] + [P(C.c_int64)] * 7
        L.clr_get_scaling.argtypes = [vp, P(C.c_double), P(C.c_double), P(C.c_double)]
        L.clr_get_history.argtypes = [vp, P(C.c_double), C.c_int32, P(C.c_int32)]
        L.clr_set_stream.argtypes = [vp, vp]
        L.clr_free.argtypes = [vp]
        L.clr_free.restype = None
        L.clr_error_string.restype = C.c_char_p
        L.clr_status_string.restype = C.c_char_p
        L.clr_last_cuda_error.restype = C.c_char_p
        L.clr_cones_scaling.argtypes = [P(clr_cone), C.c_int32, P(C.c_double), P(C.c_double), C.c_double,
                                        P(C.c_double)]
        L.clr_cones_step_length.argtypes = [P(clr_cone), C.c_int32] + [P(C.c_double)] * 4 + [C.c_double,
                                                                                            P(C.c_double)]
        L.clr_cones_combined_ds.argtypes = [P(clr_cone), C.c_int32] + [P(C.c_double)] * 4 + [C.c_double,
                                                                                            P(C.c_double)]
        L.clr_cones_time.argtypes = [P(clr_cone), C.c_int32] + [P(C.c_double)] * 4 + [C.c_double, C.c_int32,
                                                                                     P(clr_cone_times)]
        L.clr_ldl_solve.argtypes = [P(clr_csc), P(C.c_double), P(C.c_int64), C.c_int32, C.c_double, C.c_double,
                                    P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_int32), C.c_int32]
        L.clr_dense_ldl_solve_noalloc.argtypes = [vp, vp, C.c_int32, vp, vp, vp, C.c_double, C.c_double, vp, vp]
        L.clr_probe_peaks.argtypes = [C.c_int32, vp, P(clr_peaks)]
        L.clr_solve_begin.argtypes = [vp]
        L.clr_solve_iterate.argtypes = [vp, C.c_int32, P(C.c_int32), P(C.c_int32)]
        L.clr_solve_end.argtypes = [vp]
        L.clr_batch_setup.argtypes = [P(vp), C.c_int32, P(clr_problem), P(clr_settings)]
        L.clr_batch_analyze.argtypes = [P(vp), C.c_int32, P(clr_problem), P(clr_settings)]
        L.clr_batch_size.argtypes = [vp]
        L.clr_batch_size.restype = C.c_int32
        L.clr_batch_get.argtypes = [vp, C.c_int32, P(C.c_double), P(C.c_double), P(C.c_double), P(clr_info)]
        L.clr_batch_update_qb.argtypes = [vp, C.c_int32, P(C.c_double), P(C.c_double)]
        L.clr_server_create.argtypes = [P(vp), C.c_size_t, C.c_int32, C.c_int32, P(clr_settings)]
        L.clr_server_submit.argtypes = [vp, P(clr_problem), P(C.c_uint64)]
        L.clr_server_poll.argtypes = [vp, C.c_uint64, P(C.c_double), P(C.c_double), P(C.c_double), P(clr_info)]
        L.clr_server_wait.argtypes = [vp, C.c_uint64, C.c_double, P(C.c_double), P(C.c_double), P(C.c_double),
                                      P(clr_info)]
        L.clr_server_get_stats.argtypes = [vp, P(clr_server_stats)]
        L.clr_server_destroy.argtypes = [vp]
        L.clr_autotune.argtypes = [C.c_int32, P(clr_problem), P(clr_settings), C.c_int32, C.c_char_p,
                                   P(clr_tune_result)]
        _LIB = L
    return _LIB


def _err_string(code):
    try:
        return _lib().clr_error_string(code).decode()
    except Exception:
        return "error"


def _check(rc, where):
    if rc != 0:
        raise ClrError(rc, where)


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _csc(M, keep):
    M = sp.csc_matrix(M)
    M.sort_indices()
    colptr = np.ascontiguousarray(M.indptr, dtype=np.int64)
    rowind = np.ascontiguousarray(M.indices, dtype=np.int32)
    val = np.ascontiguousarray(M.data, dtype=np.float64)
    keep += [colptr, rowind, val]
    return clr_csc(M.shape[0], M.shape[1], len(val), colptr.ctypes.data_as(C.POINTER(C.c_int64)),
                   rowind.ctypes.data_as(C.POINTER(C.c_int32)), val.ctypes.data_as(C.POINTER(C.c_double)))


def _values_on(M, pattern, upper, name):
    """Values of M in the CSC order of `pattern` (indptr, indices) given to setup:
    M is a 1-D array of nnz values, or a matrix with exactly that pattern."""
    if M is None:
        return None
    if isinstance(M, np.ndarray) and M.ndim == 1:
        v = np.ascontiguousarray(M, dtype=np.float64)
    else:
        M = sp.csc_matrix(M)
        if upper and not _is_upper(M):
            M = sp.csc_matrix(sp.triu(M))
        M.sort_indices()
        if not (np.array_equal(M.indptr, pattern[0]) and np.array_equal(M.indices, pattern[1])):
            raise ValueError("%s: the sparsity pattern differs from the one given at setup" % name)
        v = np.ascontiguousarray(M.data, dtype=np.float64)
    if len(v) != len(pattern[1]):
        raise ValueError("%s: %d values for a pattern of %d entries" % (name, len(v), len(pattern[1])))
    return v


def _pattern(c):
    n = c.ncols
    ptr = np.ctypeslib.as_array(c.colptr, shape=(n + 1,)).copy()
    idx = np.ctypeslib.as_array(c.rowind, shape=(c.nnz,)).copy() if c.nnz else np.zeros(0, np.int32)
    return ptr, idx


def _cones(cones):
    arr = (clr_cone * max(len(cones), 1))()
    for i, (t, d, a) in enumerate(cones):
        arr[i] = clr_cone(int(t), int(d), float(a))
    return arr


def clr_default_settings(factor_bits=64, **overrides):
    s = clr_settings()
    _check(_lib().clr_default_settings(C.byref(s), factor_bits), "clr_default_settings")
    for k, v in overrides.items():
        setattr(s, k, v)
    return s


def settings_dict(s):
    return {name: getattr(s, name) for name, _ in clr_settings._fields_}


class Solver:
    """Owner of one clr_solver handle."""

    def __init__(self, P_upper, q, A, b, cones, settings=None, device=True):
        keep = []
        Pc = _csc(sp.triu(sp.csc_matrix(P_upper)) if not _is_upper(P_upper) else P_upper, keep)
        Ac = _csc(A, keep)
        q = np.ascontiguousarray(q, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        self.n, self.m = len(q), len(b)
        cz = _cones(cones)
        st = settings if isinstance(settings, clr_settings) else clr_default_settings(**(settings or {}))
        self.settings = st
        h = C.c_void_p()
        fn = _lib().clr_setup if device else _lib().clr_analyze
        _check(fn(C.byref(h), C.byref(Pc), _dptr(q), C.byref(Ac), _dptr(b), cz, len(cones), C.byref(st)),
               "clr_setup" if device else "clr_analyze")
        self.h = h
        self.patterns = [(_pattern(Pc), _pattern(Ac))]

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "h", None) and self.h.value:
            _lib().clr_free(self.h)
            self.h = C.c_void_p()

    def solve(self):
        """clr_solve: run Algorithm 1 from its initial point to a stopping status;
        returns the status code (STATUS maps it to a name)."""
        _check(_lib().clr_solve(self.h), "clr_solve")
        return self.info()["status"]

    def solve_begin(self):
        """clr_solve_begin: start a solve (initial point) on the solver's stream."""
        _check(_lib().clr_solve_begin(self.h), "clr_solve_begin")

    def solve_iterate(self, k=1):
        """clr_solve_iterate: up to k IPM iterations; returns (done, iterations run)."""
        done, ran = C.c_int32(), C.c_int32()
        _check(_lib().clr_solve_iterate(self.h, int(k), C.byref(done), C.byref(ran)), "clr_solve_iterate")
        return bool(done.value), ran.value

    def solve_end(self):
        """clr_solve_end: finish the solve started by solve_begin."""
        _check(_lib().clr_solve_end(self.h), "clr_solve_end")

    def info(self):
        """The clr_info of the last solve as a dict (status, status_name,
        iterations, residuals, gap, refinement and escalation counters)."""
        inf = clr_info()
        _check(_lib().clr_get_solution(self.h, None, None, None, C.byref(inf)), "clr_get_solution")
        d = {name: getattr(inf, name) for name, _ in clr_info._fields_}
        d["status_name"] = STATUS.get(d["status"], "UNKNOWN")
        return d

    def solution(self):
        """(x, s, z, info) of the last solve, unscaled, in the caller's row order."""
        x, s, z = np.empty(self.n), np.empty(self.m), np.empty(self.m)
        inf = clr_info()
        _check(_lib().clr_get_solution(self.h, _dptr(x), _dptr(s), _dptr(z), C.byref(inf)), "clr_get_solution")
        d = {name: getattr(inf, name) for name, _ in clr_info._fields_}
        d["status_name"] = STATUS.get(d["status"], "UNKNOWN")
        return x, s, z, d

    def update_qb(self, q, b):
        """New q (n) and b (m, caller's row order); the next solve uses them."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        _check(_lib().clr_update_qb(self.h, _dptr(q), _dptr(b)), "clr_update_qb")

    def update_PA(self, P=None, A=None):
        """New values of P (upper triangle) and/or A with the patterns given at
        setup: each a matrix of that pattern or a 1-D array of its values in
        CSC order; None keeps the current values."""
        self._update_PA(0, P, A)

    def _update_PA(self, i, P, A):
        (pp, ap) = self.patterns[i]
        Pv, Av = _values_on(P, pp, True, "P"), _values_on(A, ap, False, "A")
        ptr = lambda v: None if v is None else _dptr(v)
        if i == 0 and not isinstance(self, Batch):
            _check(_lib().clr_update_PA(self.h, ptr(Pv), ptr(Av)), "clr_update_PA")
        else:
            _check(_lib().clr_batch_update_PA(self.h, i, ptr(Pv), ptr(Av)), "clr_batch_update_PA")

    def set_stream(self, stream_ptr):
        """Run the solver's work on the given CUDA stream (a cudaStream_t as an int)."""
        _check(_lib().clr_set_stream(self.h, C.c_void_p(stream_ptr)), "clr_set_stream")

    def symbolic_stats(self):
        """Sizes of the symbolic factorization (KKT order, nnz(L), factor flops,
        supernodes, levels, largest front, chosen ordering) as a dict."""
        s = clr_symbolic_stats()
        _check(_lib().clr_get_symbolic_stats(self.h, C.byref(s)), "clr_get_symbolic_stats")
        return {name: getattr(s, name) for name, _ in clr_symbolic_stats._fields_}

    def perf(self):
        """Device time by phase (init, residuals+cones, factorization, solves+steps,
        ms) and counts (factorizations, kernel launches, factor flops) as a dict."""
        s = clr_perf()
        _check(_lib().clr_get_perf(self.h, C.byref(s)), "clr_get_perf")
        return {name: getattr(s, name) for name, _ in clr_perf._fields_}

    def symbolic(self):
        """The symbolic factorization: elimination order, supernode column ranges,
        parents, front row lists and the constraint-row permutation (numpy arrays)."""
        st = self.symbolic_stats()
        N, nsn = st["kkt_dim"], st["n_supernodes"]
        L = C.POINTER(C.c_int64)
        rl = C.c_int64()
        _check(_lib().clr_get_symbolic(self.h, None, None, None, None, None, C.byref(rl), None), "clr_get_symbolic")
        perm, snp, par = np.empty(N, np.int64), np.empty(nsn + 1, np.int64), np.empty(nsn, np.int64)
        rp, rows, rowperm = np.empty(nsn + 1, np.int64), np.empty(rl.value, np.int64), np.empty(self.m, np.int64)
        ptr = lambda a: a.ctypes.data_as(L)
        _check(_lib().clr_get_symbolic(self.h, ptr(perm), ptr(snp), ptr(par), ptr(rp), ptr(rows), C.byref(rl),
                                       ptr(rowperm)), "clr_get_symbolic")
        return dict(perm=perm, sn_ptr=snp, sn_parent=par, row_ptr=rp, rows=rows, row_perm=rowperm)

    def scaling(self):
        """Equilibration of the setup: D (n), E (m, reordered rows) and the cost scale c."""
        D, E, c = np.empty(self.n), np.empty(self.m), C.c_double()
        _check(_lib().clr_get_scaling(self.h, _dptr(D), _dptr(E), C.byref(c)), "clr_get_scaling")
        return D, E, c.value

    def history(self):
        """Per-iteration log of the last solve, rows of (iter, mu, pcost, dcost, res_p,
        res_d, gap, alpha_a, sigma, alpha_c, ir_steps, tau)."""
        cap = self.settings.max_iter + 2
        out = np.zeros((cap, 12))
        rows = C.c_int32()
        _check(_lib().clr_get_history(self.h, _dptr(out), cap, C.byref(rows)), "clr_get_history")
        return out[: rows.value]


def _info_dict(inf):
    d = {name: getattr(inf, name) for name, _ in clr_info._fields_}
    d["status_name"] = STATUS.get(d["status"], "UNKNOWN")
    return d


def _settings(settings):
    return settings if isinstance(settings, clr_settings) else clr_default_settings(**(settings or {}))


class Batch(Solver):
    """A cohort of independent problems solved together (clr_batch_setup).

    problems: sequence of (P_upper, q, A, b, cones)."""

    def __init__(self, problems, settings=None, device=True):
        keep = []
        arr = (clr_problem * len(problems))()
        self.sizes = []
        pats = []
        for i, (P, q, A, b, cones) in enumerate(problems):
            Pc = _csc(sp.triu(sp.csc_matrix(P)) if not _is_upper(P) else P, keep)
            Ac = _csc(A, keep)
            q = np.ascontiguousarray(q, dtype=np.float64)
            b = np.ascontiguousarray(b, dtype=np.float64)
            cz = _cones(cones)
            keep += [Pc, Ac, q, b, cz]
            arr[i] = clr_problem(C.pointer(Pc), _dptr(q), C.pointer(Ac), _dptr(b), cz, len(cones))
            self.sizes.append((len(q), len(b)))
            pats.append((_pattern(Pc), _pattern(Ac)))
        self.n, self.m = self.sizes[0]
        st = _settings(settings)
        self.settings = st
        h = C.c_void_p()
        fn = _lib().clr_batch_setup if device else _lib().clr_batch_analyze
        _check(fn(C.byref(h), len(problems), arr, C.byref(st)), "clr_batch_setup" if device else "clr_batch_analyze")
        self.h = h
        self.patterns = pats

    def size(self):
        """Number of problems in the cohort."""
        return _lib().clr_batch_size(self.h)

    def info_of(self, i):
        """info of problem i after a solve."""
        inf = clr_info()
        _check(_lib().clr_batch_get(self.h, i, None, None, None, C.byref(inf)), "clr_batch_get")
        return _info_dict(inf)

    def solution_of(self, i):
        """(x, s, z, info) of problem i, as Solver.solution for a single problem."""
        n, m = self.sizes[i]
        x, s, z = np.empty(n), np.empty(m), np.empty(m)
        inf = clr_info()
        _check(_lib().clr_batch_get(self.h, i, _dptr(x), _dptr(s), _dptr(z), C.byref(inf)), "clr_batch_get")
        return x, s, z, _info_dict(inf)

    def update_qb_of(self, i, q, b):
        """New q and b for problem i of the cohort."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        _check(_lib().clr_batch_update_qb(self.h, i, _dptr(q), _dptr(b)), "clr_batch_update_qb")

    def update_PA_of(self, i, P=None, A=None):
        """New values of P and/or A for problem i (the patterns it was set up with)."""
        self._update_PA(i, P, A)


def clr_batch_setup(problems, settings=None):
    return Batch(problems, settings)


def clr_batch_analyze(problems, settings=None):
    return Batch(problems, settings, device=False)


def clr_autotune(problems, settings=None, iters=3, cache_path=None):
    """Pick small_front_max, amalgamation and big_front_schedule for a cohort of
    problems (sequence of (P_upper, q, A, b, cones)) by timing candidate settings
    on the device (see include/clr.h).  Returns a dict of the result."""
    reqs = [Request(*p) for p in problems]
    arr = (clr_problem * len(reqs))(*[r.prob for r in reqs])
    st = _settings(settings)
    out = clr_tune_result()
    path = cache_path.encode() if cache_path else None
    _check(_lib().clr_autotune(len(reqs), arr, C.byref(st), int(iters), path, C.byref(out)), "clr_autotune")
    return {k: getattr(out, k) for (k, _) in clr_tune_result._fields_ if k != "pad"}


class Request:
    """Marshalled arguments of one problem, ready to submit (built ahead of time)."""

    def __init__(self, P_upper, q, A, b, cones):
        self.keep = []
        self.Pc = _csc(sp.triu(sp.csc_matrix(P_upper)) if not _is_upper(P_upper) else P_upper, self.keep)
        self.Ac = _csc(A, self.keep)
        self.q = np.ascontiguousarray(q, dtype=np.float64)
        self.b = np.ascontiguousarray(b, dtype=np.float64)
        self.cz = _cones(cones)
        self.n, self.m = len(self.q), len(self.b)
        self.prob = clr_problem(C.pointer(self.Pc), _dptr(self.q), C.pointer(self.Ac), _dptr(self.b), self.cz,
                                len(cones))


class Server:
    """clr_server_*: continuous-batching request loop on the current device."""

    def __init__(self, device_bytes=8 << 30, max_cohort=256, max_active=4, settings=None):
        st = _settings(settings)
        self.settings = st
        h = C.c_void_p()
        _check(_lib().clr_server_create(C.byref(h), int(device_bytes), int(max_cohort), int(max_active),
                                        C.byref(st)), "clr_server_create")
        self.h = h
        self.sizes = {}

    def submit(self, req):
        """Queue a Request (deep-copied by the server); returns its ticket."""
        t = C.c_uint64()
        _check(_lib().clr_server_submit(self.h, C.byref(req.prob), C.byref(t)), "clr_server_submit")
        self.sizes[t.value] = (req.n, req.m)
        return t.value

    def _result(self, fn, ticket, *extra):
        n, m = self.sizes[ticket]
        x, s, z = np.empty(n), np.empty(m), np.empty(m)
        inf = clr_info()
        rc = fn(self.h, C.c_uint64(ticket), *extra, _dptr(x), _dptr(s), _dptr(z), C.byref(inf))
        if rc in (-6, -7):  # CLR_E_TIMEOUT, CLR_E_AGAIN
            return None
        self.sizes.pop(ticket, None)
        _check(rc, "clr_server_poll")
        return x, s, z, _info_dict(inf)

    def poll(self, ticket):
        """(x, s, z, info) of a finished request, or None while it runs."""
        return self._result(_lib().clr_server_poll, ticket)

    def wait(self, ticket, timeout_s=60.0):
        """Block until the request finishes (None after timeout_s seconds)."""
        return self._result(_lib().clr_server_wait, ticket, C.c_double(timeout_s))

    def stats(self):
        """Server counters (requests, cohorts, device memory in use and peak) as a dict."""
        s = clr_server_stats()
        _check(_lib().clr_server_get_stats(self.h, C.byref(s)), "clr_server_get_stats")
        return {name: getattr(s, name) for name, _ in clr_server_stats._fields_}

    def close(self):
        """Finish the requests in flight and release the server."""
        if getattr(self, "h", None) and self.h.value:
            _lib().clr_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        self.close()


def _is_upper(P):
    P = sp.coo_matrix(P)
    return bool(np.all(P.row <= P.col))


def clr_setup(P_upper, q, A, b, cones, settings=None):
    """Set up a solver on the current GPU (host analysis, then device buffers)."""
    return Solver(P_upper, q, A, b, cones, settings, device=True)


def clr_analyze(P_upper, q, A, b, cones, settings=None):
    """The host analysis only (validation, equilibration, ordering, symbolic
    factorization); no device memory, usable without a GPU."""
    return Solver(P_upper, q, A, b, cones, settings, device=False)


def clr_cones_scaling(cones, s, z, mu):
    s = np.ascontiguousarray(s, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    H = np.zeros(sum(int(d) * int(d) for (_, d, _) in cones))
    _check(_lib().clr_cones_scaling(_cones(cones), len(cones), _dptr(s), _dptr(z), float(mu), _dptr(H)),
           "clr_cones_scaling")
    out, off = [], 0
    for (_, d, _) in cones:
        out.append(H[off:off + d * d].reshape(d, d))
        off += d * d
    return out


def clr_cones_step_length(cones, s, z, ds, dz, alpha_max=1.0):
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (s, z, ds, dz)]
    a = C.c_double()
    _check(_lib().clr_cones_step_length(_cones(cones), len(cones), *[_dptr(v) for v in arrs], float(alpha_max),
                                        C.byref(a)), "clr_cones_step_length")
    return a.value


def clr_cones_combined_ds(cones, s, z, ds_a, dz_a, sigma_mu):
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (s, z, ds_a, dz_a)]
    out = np.zeros(len(arrs[0]))
    _check(_lib().clr_cones_combined_ds(_cones(cones), len(cones), *[_dptr(v) for v in arrs], float(sigma_mu),
                                        _dptr(out)), "clr_cones_combined_ds")
    return out


def clr_cones_time(cones, s, z, ds, dz, mu, reps=10):
    """Mean device ms per call of the scaling, step-length and combined-d_s
    kernels on one cone list (see include/clr.h)."""
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (s, z, ds, dz)]
    out = clr_cone_times()
    _check(_lib().clr_cones_time(_cones(cones), len(cones), *[_dptr(v) for v in arrs], float(mu), int(reps),
                                 C.byref(out)), "clr_cones_time")
    return {k: getattr(out, k) for (k, _) in clr_cone_times._fields_}


def clr_ldl_solve(K_lower, signs, rhs, order=None, factor_bits=64, dyn_reg_eps=1e-13, dyn_reg_delta=2e-7,
                  big_front_schedule=1):
    keep = []
    Kc = _csc(sp.tril(sp.csc_matrix(K_lower)), keep)
    signs = np.ascontiguousarray(signs, dtype=np.float64)
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    N = len(rhs)
    x, D = np.zeros(N), np.zeros(N)
    hits = C.c_int32()
    ordp = None
    if order is not None:
        order = np.ascontiguousarray(order, dtype=np.int64)
        ordp = order.ctypes.data_as(C.POINTER(C.c_int64))
    _check(_lib().clr_ldl_solve(C.byref(Kc), _dptr(signs), ordp, factor_bits, dyn_reg_eps, dyn_reg_delta, _dptr(rhs),
                                _dptr(x), _dptr(D), C.byref(hits), int(big_front_schedule)), "clr_ldl_solve")
    return x, D, hits.value


class clr_peaks(C.Structure):
    _fields_ = [("fp64_fma_tflops", C.c_double), ("fp32_fma_tflops", C.c_double), ("tf32_tc_tflops", C.c_double),
                ("bf16_tc_tflops", C.c_double), ("fp64_ms", C.c_double), ("fp32_ms", C.c_double),
                ("tf32_ms", C.c_double), ("bf16_ms", C.c_double), ("sms", C.c_int32), ("tc_timeouts", C.c_int32)]


def clr_probe_peaks(reps=5, stream_ptr=None):
    """FP64 / FP32 FMA and tcgen05 TF32 / BF16 tensor throughput (TFLOP/s) of
    the current GPU, measured by the library's probe kernels (see include/clr.h)."""
    out = clr_peaks()
    _check(_lib().clr_probe_peaks(int(reps), C.c_void_p(stream_ptr), C.byref(out)), "clr_probe_peaks")
    return {k: getattr(out, k) for (k, _) in clr_peaks._fields_}


def clr_dense_ldl_solve_noalloc(K_ptr, signs_ptr, N, rhs_ptr, x_ptr, D_ptr=None, dyn_reg_eps=1e-13,
                                dyn_reg_delta=2e-7, hits_ptr=None, stream_ptr=None):
    """Device-pointer call of the allocation-free dense LDL^T solve (pointers as ints)."""
    _check(_lib().clr_dense_ldl_solve_noalloc(C.c_void_p(K_ptr), C.c_void_p(signs_ptr), int(N), C.c_void_p(rhs_ptr),
                                              C.c_void_p(x_ptr), C.c_void_p(D_ptr), float(dyn_reg_eps),
                                              float(dyn_reg_delta), C.c_void_p(hits_ptr), C.c_void_p(stream_ptr)),
           "clr_dense_ldl_solve_noalloc")
