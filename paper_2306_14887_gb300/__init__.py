"""Python binding of the tnbp C ABI (include/tnbp.h): argument marshalling only.

Every step of the simulation runs in the CUDA library ``libtnbp.so`` built
in-tree for sm_103a; this module loads it with ctypes, passes plain pointers
and sizes, and binds the library's device allocator to PyTorch's caching
allocator.  There is no CPU fallback: if the library is missing or cannot
load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtnbp.so")

TN_OK = 0
STATUS = {0: "TN_OK", -1: "TN_EINVAL", -2: "TN_ENOMEM", -3: "TN_ENOTCONVERGED",
          -4: "TN_ENUMERIC", -5: "TN_ETIMEOUT", -6: "TN_ECUDA", -7: "TN_EAGAIN",
          -8: "TN_EUNSUPPORTED"}
PRECISIONS = {"fp32": 0, "tf32": 1, "bf16": 2, "bf16x3": 3, "tf32x3": 4}
SOLVES = {"auto": 0, "fp64": 1, "shared": 2, "refined": 3}
KERNELS = {"auto": 0, "tile": 1}

#: every symbol include/tnbp.h declares
EXPORTS = ["tn_create", "tn_destroy", "tn_apply_floquet", "tn_apply_clifford_dagger",
           "tn_bp_converge", "tn_expect", "tn_expect_z_all", "tn_get_stats", "tn_get_site",
           "tn_set_site", "tn_get_message", "tn_set_message", "tn_footprint",
           "tn_footprint_estimate", "tn_heavy_hex", "tn_clifford_reduce", "tn_profile_enable",
           "tn_profile_read", "tn_profile_class_name", "tn_truncation_solve",
           "tn_truncation_solve_noalloc", "tn_truncation_solve_ex", "tn_last_error",
           "tn_version", "tn_apply_floquet_field", "tn_server_create", "tn_server_submit",
           "tn_server_poll", "tn_server_wait", "tn_server_get_stats", "tn_server_destroy",
           "tn_server_poll_ex", "tn_server_wait_ex",
           "tn_bond_spectrum", "tn_entanglement_entropy", "tn_state_size", "tn_save_state",
           "tn_load_state", "tn_chi_extrapolate", "tn_vidal_gauge", "tn_get_gamma",
           "tn_bp_error", "tn_graph_info", "tn_selftest_bounded_wait", "tn_bp_components",
           "tn_autotune", "tn_autotune_apply"]


class TNError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class tn_graph(C.Structure):
    _fields_ = [("n_vertices", C.c_int32), ("n_edges", C.c_int32),
                ("edges", C.POINTER(C.c_int32)), ("colour", C.POINTER(C.c_uint8)),
                ("periodic", C.c_int32)]


class tn_config(C.Structure):
    _fields_ = [("chi", C.c_int32), ("prec", C.c_int32), ("bp_tol", C.c_double),
                ("bp_max_iters", C.c_int32), ("svd_cutoff", C.c_double), ("seed", C.c_uint64),
                ("solve", C.c_int32), ("kernels", C.c_int32),
                ("solve_tol", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class tn_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class tn_stats(C.Structure):
    _fields_ = [("steps_done", C.c_int32), ("bp_iters_last", C.c_int32),
                ("bp_iters_total", C.c_int32), ("bp_residual_last", C.c_double),
                ("discarded_max", C.c_double), ("discarded_sum", C.c_double),
                ("kernel_launches", C.c_int64), ("tma_launches", C.c_int64),
                ("solve_edges", C.c_int64), ("solve_sweeps", C.c_int64),
                ("solve_sweeps_max", C.c_int64)]


class tn_profile(C.Structure):
    _fields_ = [("n_classes", C.c_int32), ("launches", C.c_int64 * 16), ("ms", C.c_double * 16),
                ("flops", C.c_double * 16), ("bytes", C.c_double * 16)]


class tn_pauli(C.Structure):
    _fields_ = [("weight", C.c_int32), ("sites", C.POINTER(C.c_int32)),
                ("paulis", C.c_char_p), ("sign", C.c_int8)]


class tn_server_config(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_slots", C.c_int32), ("device", C.c_int32),
                ("policy", C.c_int32)]


class tn_job(C.Structure):
    _fields_ = [("graph", tn_graph), ("cfg", tn_config), ("theta_h", C.c_double),
                ("steps", C.c_int32), ("ops", C.c_void_p), ("n_ops", C.c_int32),
                ("ops_method", C.c_int32)]


class tn_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_vertices", C.c_int32), ("steps_done", C.c_int32),
                ("queue_s", C.c_double), ("latency_s", C.c_double)]


class tn_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("resident", C.c_int32), ("peak_resident", C.c_int32), ("queued", C.c_int32),
                ("used_bytes", C.c_size_t), ("peak_bytes", C.c_size_t),
                ("budget_bytes", C.c_size_t)]


_lib = None


def lib():
    """Load libtnbp.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing; run paper_2306_14887_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, dp = C.c_void_p, C.c_int32, C.POINTER(C.c_double)
        L.tn_create.argtypes = [C.POINTER(tn_graph), C.POINTER(tn_config),
                                C.POINTER(tn_allocator), vp, C.POINTER(vp)]
        L.tn_destroy.argtypes = [vp]
        L.tn_apply_floquet.argtypes = [vp, C.c_double, i32]
        L.tn_apply_clifford_dagger.argtypes = [vp, i32]
        L.tn_bp_converge.argtypes = [vp, C.c_double, i32, C.POINTER(i32), dp]
        L.tn_autotune.argtypes = [vp, i32, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]
        L.tn_autotune_apply.argtypes = [vp, C.c_char_p, C.POINTER(i32)]
        L.tn_bp_components.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), dp, i32, C.POINTER(i32)]
        L.tn_expect.argtypes = [vp, C.POINTER(tn_pauli), i32, i32, dp]
        L.tn_expect_z_all.argtypes = [vp, dp]
        L.tn_get_stats.argtypes = [vp, C.POINTER(tn_stats)]
        fp = C.POINTER(C.c_float)
        L.tn_get_site.argtypes = [vp, i32, fp, C.c_size_t]
        L.tn_set_site.argtypes = [vp, i32, fp, C.c_size_t]
        L.tn_get_message.argtypes = [vp, i32, i32, fp, C.c_size_t]
        L.tn_set_message.argtypes = [vp, i32, i32, fp, C.c_size_t]
        L.tn_footprint.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.tn_footprint_estimate.argtypes = [C.POINTER(tn_graph), C.POINTER(tn_config),
                                            C.POINTER(C.c_size_t)]
        L.tn_heavy_hex.argtypes = [i32, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                   C.POINTER(C.c_uint8), i32]
        L.tn_clifford_reduce.argtypes = [C.POINTER(tn_graph), C.POINTER(tn_pauli), i32,
                                         C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.tn_profile_enable.argtypes = [vp, i32]
        L.tn_profile_read.argtypes = [vp, C.POINTER(tn_profile)]
        L.tn_profile_class_name.argtypes = [i32]
        L.tn_profile_class_name.restype = C.c_char_p
        L.tn_truncation_solve.argtypes = [vp, vp, vp, i32, i32, i32, C.c_double, vp]
        L.tn_truncation_solve_noalloc.argtypes = [vp, vp, vp, i32, i32, i32, C.c_double, vp]
        L.tn_truncation_solve_ex.argtypes = [vp, vp, vp, i32, i32, i32, C.c_double, i32, vp]
        L.tn_apply_floquet_field.argtypes = [vp, dp, i32]
        L.tn_bond_spectrum.argtypes = [vp, i32, dp]
        L.tn_state_size.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.tn_save_state.argtypes = [vp, vp, C.c_size_t]
        L.tn_load_state.argtypes = [vp, vp, C.c_size_t]
        L.tn_entanglement_entropy.argtypes = [vp, i32, dp]
        L.tn_server_create.argtypes = [C.POINTER(tn_server_config), C.POINTER(vp)]
        L.tn_server_submit.argtypes = [vp, C.POINTER(tn_job), C.POINTER(C.c_uint64)]
        L.tn_server_poll.argtypes = [vp, C.c_uint64, dp, C.POINTER(tn_result)]
        L.tn_server_wait.argtypes = [vp, C.c_uint64, C.c_double, dp, C.POINTER(tn_result)]
        L.tn_server_poll_ex.argtypes = [vp, C.c_uint64, dp, dp, C.POINTER(tn_result)]
        L.tn_server_wait_ex.argtypes = [vp, C.c_uint64, C.c_double, dp, dp, C.POINTER(tn_result)]
        L.tn_server_get_stats.argtypes = [vp, C.POINTER(tn_server_stats)]
        L.tn_server_destroy.argtypes = [vp]
        L.tn_chi_extrapolate.argtypes = [dp, dp, i32, i32, dp, dp, dp]
        L.tn_vidal_gauge.argtypes = [vp, dp]
        L.tn_selftest_bounded_wait.argtypes = [vp, C.POINTER(i32)]
        L.tn_bp_error.argtypes = [vp, i32, dp, dp, i32, C.POINTER(i32)]
        L.tn_graph_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                    C.POINTER(i32), i32]
        L.tn_get_gamma.argtypes = [vp, i32, C.POINTER(C.c_float), C.c_size_t]
        L.tn_last_error.restype = C.c_char_p
        L.tn_version.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("tn_last_error", "tn_version", "tn_profile_class_name"):
                getattr(L, name).restype = C.c_int32
        _lib = L
    return _lib


def _check(status):
    if status != TN_OK:
        raise TNError(status, lib().tn_last_error().decode())
    return status


def heavy_hex(rows, cols):
    """(n_vertices, edges [m, 2] int32, colours [m] uint8) from the library's generator."""
    L = lib()
    n, m = C.c_int32(), C.c_int32()
    _check(L.tn_heavy_hex(rows, cols, C.byref(n), C.byref(m), None, None, 0))
    edges = np.zeros((m.value, 2), dtype=np.int32)
    cols_ = np.zeros(m.value, dtype=np.uint8)
    _check(L.tn_heavy_hex(rows, cols, C.byref(n), C.byref(m),
                          edges.ctypes.data_as(C.POINTER(C.c_int32)),
                          cols_.ctypes.data_as(C.POINTER(C.c_uint8)), m.value))
    return n.value, edges, cols_


def clifford_reduce(n, edges, ops, sign=1, max_steps=32, colours=None):
    """(site, n', sign) with ops = sign * U^n'(pi/2) Z_site U^n'(pi/2)^dagger (host-only)."""
    g, _keep = _graph_struct(n, edges, colours)
    sites = np.array(sorted(ops), dtype=np.int32)
    labels = "".join(ops[int(q)] for q in sites).encode()
    p = tn_pauli(len(sites), sites.ctypes.data_as(C.POINTER(C.c_int32)), labels, int(sign))
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().tn_clifford_reduce(C.byref(g), C.byref(p), int(max_steps), C.byref(a),
                                    C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def truncation_solve(gram, dmat, s_out, n_edges, chi, sign=1, svd_cutoff=0.0, stream=0,
                     solve="fp64"):
    """Standalone truncation solve on device buffers (raw pointers as ints)."""
    _check(lib().tn_truncation_solve_ex(C.c_void_p(gram), C.c_void_p(dmat), C.c_void_p(s_out),
                                        int(n_edges), int(chi), int(sign), float(svd_cutoff),
                                        SOLVES[solve], C.c_void_p(stream)))


def truncation_solve_noalloc(gram, dmat, s_out, n_edges, chi, sign=1, svd_cutoff=0.0, stream=0):
    """tn_truncation_solve without device allocation: for callers whose device
    memory is owned by someone else; workspace is a fixed 16 MiB array in the
    library (see include/tnbp.h for the size limit and the sharing rules)."""
    _check(lib().tn_truncation_solve_noalloc(C.c_void_p(gram), C.c_void_p(dmat),
                                             C.c_void_p(s_out), int(n_edges), int(chi),
                                             int(sign), float(svd_cutoff), C.c_void_p(stream)))


def _graph_struct(n, edges, colours):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    g = tn_graph()
    g.n_vertices = int(n)
    g.n_edges = len(e) // 2
    g.edges = e.ctypes.data_as(C.POINTER(C.c_int32))
    keep = [e]
    if colours is not None:
        c = np.ascontiguousarray(np.asarray(colours, dtype=np.uint8))
        g.colour = c.ctypes.data_as(C.POINTER(C.c_uint8))
        keep.append(c)
    else:
        g.colour = C.POINTER(C.c_uint8)()
    g.periodic = 0
    return g, keep


def _config(chi, prec, bp_tol, bp_max_iters, svd_cutoff, solve="auto", kernels="auto",
            solve_tol=0.0):
    c = tn_config()
    c.solve_tol = float(solve_tol)
    c.solve = SOLVES[solve] if isinstance(solve, str) else int(solve)
    c.kernels = KERNELS[kernels] if isinstance(kernels, str) else int(kernels)
    c.chi = int(chi)
    c.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    c.bp_tol = float(bp_tol)
    c.bp_max_iters = int(bp_max_iters)
    c.svd_cutoff = float(svd_cutoff)
    c.seed = 0
    return c


def footprint_estimate(n, edges, colours, chi, prec="fp32"):
    g, _keep = _graph_struct(n, edges, colours)
    cfg = _config(chi, prec, 1e-10, 1, 0.0)
    out = C.c_size_t()
    _check(lib().tn_footprint_estimate(C.byref(g), C.byref(cfg), C.byref(out)))
    return out.value


class TNState:
    """A tensor-network state on one graph, resident on the current CUDA device."""

    def __init__(self, n, edges, colours=None, chi=8, prec="fp32", bp_tol=1e-10,
                 bp_max_iters=1000, svd_cutoff=0.0, stream=None, torch_allocator=True,
                 solve="auto", kernels="auto", solve_tol=0.0):
        import torch
        self._torch = torch
        L = lib()
        self.n = int(n)
        self.edges = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
        self.chi = int(chi)
        g, self._keep = _graph_struct(n, edges, colours)
        cfg = _config(chi, prec, bp_tol, bp_max_iters, svd_cutoff, solve, kernels, solve_tol)
        if stream is None:
            # a stream of its own: the library captures its BP sweep as a CUDA
            # graph, which the legacy default stream does not allow
            stream = torch.cuda.Stream()
        self._stream = stream
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._sp = sp
        self._alloc = None
        if torch_allocator:
            dev = torch.cuda.current_device()

            def _a(size, ctx, st):
                try:
                    return torch.cuda.caching_allocator_alloc(int(size), dev, int(st or 0))
                except Exception:
                    return None

            def _f(ptr, size, ctx, st):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._cb = (ALLOC_FN(_a), FREE_FN(_f))
            self._alloc = tn_allocator(self._cb[0], self._cb[1], None)
        h = C.c_void_p()
        _check(L.tn_create(C.byref(g), C.byref(cfg),
                           C.byref(self._alloc) if self._alloc is not None else None,
                           C.c_void_p(sp), C.byref(h)))
        self._h = h

    # ------------------------------------------------------------------ life
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().tn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -------------------------------------------------------------- evolution
    def apply_floquet(self, theta, steps, check=True):
        s = lib().tn_apply_floquet(self._h, float(theta), int(steps))
        if check and s not in (TN_OK, -3):
            _check(s)
        return s

    def apply_floquet_field(self, thetas, steps, check=True):
        """U with a kick angle per vertex (thetas: n values)."""
        th = np.ascontiguousarray(thetas, dtype=np.float64).reshape(-1)
        if th.size != self.n:
            raise ValueError(f"need {self.n} angles, got {th.size}")
        s = lib().tn_apply_floquet_field(self._h, th.ctypes.data_as(C.POINTER(C.c_double)),
                                         int(steps))
        if check and s not in (TN_OK, -3):
            _check(s)
        return s

    def apply_clifford_dagger(self, steps):
        s = lib().tn_apply_clifford_dagger(self._h, int(steps))
        if s not in (TN_OK, -3):
            _check(s)
        return s

    def bp_converge(self, tol=1e-10, max_iters=1000):
        it, res = C.c_int32(), C.c_double()
        s = lib().tn_bp_converge(self._h, float(tol), int(max_iters), C.byref(it), C.byref(res))
        if s not in (TN_OK, -3):
            _check(s)
        return it.value, res.value, s

    def autotune(self, reps=5):
        """Time the split-K counts of the BP-sweep launches (tn_autotune) and
        keep the fastest; returns the table as text."""
        n = C.c_size_t()
        buf = C.create_string_buffer(1 << 20)
        _check(lib().tn_autotune(self._h, int(reps), buf, len(buf), C.byref(n)))
        if n.value >= len(buf):
            raise RuntimeError("autotune table longer than its buffer")
        return buf.value.decode()

    def apply_tuning(self, table):
        """Apply a table from autotune (this or another handle); returns the
        number of rows applied."""
        k = C.c_int32()
        _check(lib().tn_autotune_apply(self._h, table.encode(), C.byref(k)))
        return k.value

    def save_tuning(self, path, reps=5):
        """Autotune and write the table to a text file."""
        table = self.autotune(reps)
        with open(path, "w") as f:
            f.write(table)
        return table

    def load_tuning(self, path):
        with open(path) as f:
            return self.apply_tuning(f.read())

    def bp_components(self):
        """(comp_of_vertex, sweeps, residuals) of the last BP iteration, per
        connected component (instance of a disjoint union)."""
        nc = C.c_int32()
        _check(lib().tn_bp_components(self._h, None, None, None, 0, C.byref(nc)))
        comp = np.zeros(self.n, dtype=np.int32)
        sw = np.zeros(max(1, nc.value), dtype=np.int32)
        res = np.zeros(max(1, nc.value), dtype=np.float64)
        _check(lib().tn_bp_components(self._h, comp.ctypes.data_as(C.POINTER(C.c_int32)),
                                      sw.ctypes.data_as(C.POINTER(C.c_int32)),
                                      res.ctypes.data_as(C.POINTER(C.c_double)), nc.value,
                                      C.byref(nc)))
        return comp, sw[:nc.value], res[:nc.value]

    # ---------------------------------------------------------- expectations
    def expect_z_all(self):
        out = np.zeros(self.n, dtype=np.float64)
        _check(lib().tn_expect_z_all(self._h, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def expect(self, strings, method=1):
        """strings: list of (dict {site: 'X'|'Y'|'Z'}, sign)."""
        arr = (tn_pauli * len(strings))()
        keep = []
        for i, (ops, sign) in enumerate(strings):
            sites = np.array(sorted(ops), dtype=np.int32)
            labels = "".join(ops[int(q)] for q in sites).encode()
            keep.append((sites, labels))
            arr[i].weight = len(sites)
            arr[i].sites = sites.ctypes.data_as(C.POINTER(C.c_int32))
            arr[i].paulis = labels
            arr[i].sign = int(sign)
        out = np.zeros(len(strings), dtype=np.float64)
        _check(lib().tn_expect(self._h, arr, len(strings), int(method),
                               out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def save_state(self):
        """Host image (bytes) of the state: site tensors, messages, bond spectra."""
        n = C.c_size_t()
        _check(lib().tn_state_size(self._h, C.byref(n)))
        buf = (C.c_ubyte * n.value)()
        _check(lib().tn_save_state(self._h, buf, n.value))
        return bytes(buf)

    def load_state(self, image):
        buf = (C.c_ubyte * len(image)).from_buffer_copy(image)
        _check(lib().tn_load_state(self._h, buf, len(image)))

    def bond_spectrum(self, e):
        out = np.zeros(self.chi, dtype=np.float64)
        _check(lib().tn_bond_spectrum(self._h, int(e), out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def entanglement_entropy(self, e):
        out = C.c_double()
        _check(lib().tn_entanglement_entropy(self._h, int(e), C.byref(out)))
        return out.value

    def stats(self):
        s = tn_stats()
        _check(lib().tn_get_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in tn_stats._fields_}

    def profile_enable(self, on=True):
        _check(lib().tn_profile_enable(self._h, 1 if on else 0))

    def profile(self):
        """{class name: {launches, ms, flops, bytes}} since profile_enable."""
        p = tn_profile()
        _check(lib().tn_profile_read(self._h, C.byref(p)))
        out = {}
        for c in range(p.n_classes):
            name = lib().tn_profile_class_name(c).decode()
            out[name] = {"launches": p.launches[c], "ms": p.ms[c], "flops": p.flops[c],
                         "bytes": p.bytes[c]}
        return out

    def footprint(self):
        out = C.c_size_t()
        _check(lib().tn_footprint(self._h, C.byref(out)))
        return out.value

    # ------------------------------------------------------------ state I/O
    def degree(self, v):
        return int(np.sum(self.edges == v))

    def get_site(self, v):
        d = self.degree(v)
        buf = np.zeros(4 * self.chi ** d, dtype=np.float32)
        _check(lib().tn_get_site(self._h, int(v), buf.ctypes.data_as(C.POINTER(C.c_float)),
                                 buf.size))
        z = buf[0::2] + 1j * buf[1::2]
        return z.reshape((2,) + (self.chi,) * d)

    def vidal_gauge(self):
        """lambda_e per edge ([n_edges, chi], decreasing, unit 2-norm) of the
        Vidal gauge from the current messages; Gamma_v then via get_gamma."""
        lam = np.zeros((len(self.edges), self.chi), dtype=np.float64)
        _check(lib().tn_vidal_gauge(self._h, lam.ctypes.data_as(C.POINTER(C.c_double))))
        return lam

    def bp_error(self, e):
        """(1 - sqrt(index of separability), singular values of the edge
        environment) of edge e in the symmetric gauge (tn_bp_error)."""
        err = C.c_double()
        cap = self.chi * self.chi
        sv = np.zeros(cap, dtype=np.float64)
        nsv = C.c_int32()
        _check(lib().tn_bp_error(self._h, int(e), C.byref(err),
                                 sv.ctypes.data_as(C.POINTER(C.c_double)), cap, C.byref(nsv)))
        return err.value, sv[:nsv.value]

    def get_gamma(self, v):
        d = self.degree(v)
        buf = np.zeros(4 * self.chi ** d, dtype=np.float32)
        _check(lib().tn_get_gamma(self._h, int(v), buf.ctypes.data_as(C.POINTER(C.c_float)),
                                  buf.size))
        return (buf[0::2] + 1j * buf[1::2]).reshape((2,) + (self.chi,) * d)

    def set_site(self, v, t):
        t = np.asarray(t, dtype=np.complex64).reshape(-1)
        buf = np.empty(2 * t.size, dtype=np.float32)
        buf[0::2], buf[1::2] = t.real, t.imag
        _check(lib().tn_set_site(self._h, int(v), buf.ctypes.data_as(C.POINTER(C.c_float)),
                                 buf.size))

    def get_message(self, e, src):
        buf = np.zeros(2 * self.chi ** 2, dtype=np.float32)
        _check(lib().tn_get_message(self._h, int(e), int(src),
                                    buf.ctypes.data_as(C.POINTER(C.c_float)), buf.size))
        return (buf[0::2] + 1j * buf[1::2]).reshape(self.chi, self.chi)

    def set_message(self, e, src, m):
        m = np.asarray(m, dtype=np.complex64).reshape(-1)
        buf = np.empty(2 * m.size, dtype=np.float32)
        buf[0::2], buf[1::2] = m.real, m.imag
        _check(lib().tn_set_message(self._h, int(e), int(src),
                                    buf.ctypes.data_as(C.POINTER(C.c_float)), buf.size))


def batch_union(instances):
    """Disjoint union of graphs [(n, edges, colours), ...] -> (n, edges, colours,
    offsets): instance i's vertex v is vertex offsets[i] + v of the union.  Many
    instances evolve as one handle (one set of launches per contraction) with
    TNState.apply_floquet_field carrying each instance's kick angle."""
    offs, es, cs = [], [], []
    n = 0
    for (ni, ei, ci) in instances:
        offs.append(n)
        e = np.asarray(ei, dtype=np.int32).reshape(-1, 2)
        es.append(e + n)
        cs.append(np.asarray(ci, dtype=np.uint8).reshape(-1))
        n += int(ni)
    return n, np.concatenate(es), np.concatenate(cs), offs


class Batch:
    """Many independent instances of uneven size, kick angle and chi evolved
    together: one disjoint-union handle per chi (BP and the simple update never
    couple components, and the BP stop rule acts on each component alone, so
    an instance's result does not depend on its batch-mates), the handles
    driven concurrently by one host thread and CUDA stream each, so that the
    groups' kernels overlap on the device.

    instances: list of (n, edges, colours, chi, theta_h)."""

    def __init__(self, instances, prec="tf32", solve="auto", **kw):
        self.sizes = [int(inst[0]) for inst in instances]
        groups = {}
        for i, inst in enumerate(instances):
            groups.setdefault(int(inst[3]), []).append(i)
        self.groups = []
        try:
            for chi, idx in sorted(groups.items()):
                n, e, c, offs = batch_union([tuple(instances[i][:3]) for i in idx])
                th = np.concatenate([np.full(self.sizes[i], float(instances[i][4])) for i in idx])
                st = TNState(n, e, c, chi=chi, prec=prec, solve=solve, **kw)
                self.groups.append((chi, idx, offs, th, st))
        except Exception:
            self.close()
            raise

    def evolve(self, steps):
        """`steps` Floquet steps of every instance (each group's handle on its
        own host thread; the library releases the interpreter lock)."""
        import threading
        errs = []

        def run(g):
            try:
                g[4].apply_floquet_field(g[3], steps)
            except Exception as ex:  # re-raised on the caller's thread
                errs.append(ex)

        threads = [threading.Thread(target=run, args=(g,)) for g in self.groups]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if errs:
            raise errs[0]

    def autotune(self, reps=3):
        """Split-K autotuning (tn_autotune) of every group's union handle on
        its current state; returns {chi: table}."""
        return {g[0]: g[4].autotune(reps) for g in self.groups}

    def expect_z(self):
        """<Z_v> of every instance, in input order."""
        out = [None] * len(self.sizes)
        for _chi, idx, offs, _th, st in self.groups:
            z = st.expect_z_all()
            for i, off in zip(idx, offs):
                out[i] = z[off:off + self.sizes[i]]
        return out

    def bp_sweeps(self):
        """Sweeps of every instance in its last BP iteration, in input order."""
        out = np.zeros(len(self.sizes), dtype=np.int32)
        for _chi, idx, offs, _th, st in self.groups:
            comp, sw, _res = st.bp_components()
            for i, off in zip(idx, offs):
                # an instance's largest component count (a connected instance has one)
                out[i] = sw[np.unique(comp[off:off + self.sizes[i]])].max()
        return out

    def close(self):
        for g in self.groups:
            g[4].close()
        self.groups = []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Continuous-batching job server on one device (see tn_server_* in tnbp.h)."""

    POLICIES = {"fifo": 0, "shortest": 1}

    def __init__(self, slots=4, hbm_budget=0, device=None, policy="fifo"):
        """policy: "fifo" (oldest queued job first) or "shortest" (least
        estimated work first among the jobs that fit)."""
        import torch
        cfg = tn_server_config()
        cfg.hbm_budget = int(hbm_budget)
        cfg.max_slots = int(slots)
        cfg.policy = self.POLICIES[policy]
        cfg.device = int(torch.cuda.current_device() if device is None else device)
        h = C.c_void_p()
        _check(lib().tn_server_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self._n = {}

    def submit(self, n, edges, colours, chi, theta, steps, prec="fp32", bp_tol=1e-10,
               bp_max_iters=1000, svd_cutoff=0.0, solve="auto", ops=None, method=0):
        """Queue a job; ops: optional list of (dict {site: 'X'|'Y'|'Z'}, sign)
        strings evaluated after the steps by tn_expect's method (0 region, 1
        extended evolution); their values come back in info["ops"]."""
        g, keep = _graph_struct(n, edges, colours)
        job = tn_job()
        job.graph = g
        job.cfg = _config(chi, prec, bp_tol, bp_max_iters, svd_cutoff, solve)
        job.theta_h = float(theta)
        job.steps = int(steps)
        ops = list(ops or [])
        arr = (tn_pauli * max(1, len(ops)))()
        hold = []
        for i, (o, sign) in enumerate(ops):
            sites = np.array(sorted(o), dtype=np.int32)
            labels = "".join(o[int(q)] for q in sites).encode()
            hold.append((sites, labels))
            arr[i].weight = len(sites)
            arr[i].sites = sites.ctypes.data_as(C.POINTER(C.c_int32))
            arr[i].paulis = labels
            arr[i].sign = int(sign)
        job.ops = C.cast(arr, C.c_void_p) if ops else None
        job.n_ops = len(ops)
        job.ops_method = int(method)
        t = C.c_uint64()
        _check(lib().tn_server_submit(self._h, C.byref(job), C.byref(t)))
        del keep, hold
        self._n[t.value] = (int(n), len(ops))
        return t.value

    def _take(self, fn, ticket, *extra):
        n, n_ops = self._n[ticket]
        z = np.zeros(n, dtype=np.float64)
        vals = np.zeros(max(1, n_ops), dtype=np.float64)
        info = tn_result()
        st = fn(self._h, C.c_uint64(ticket), *extra,
                z.ctypes.data_as(C.POINTER(C.c_double)),
                vals.ctypes.data_as(C.POINTER(C.c_double)), C.byref(info))
        if st == -7:  # TN_EAGAIN
            return None
        del self._n[ticket]
        _check(st if st != -3 else 0)
        return z, {"status": info.status, "steps_done": info.steps_done,
                   "queue_s": info.queue_s, "latency_s": info.latency_s,
                   "ops": vals[:n_ops].copy()}

    def poll(self, ticket):
        """None while queued or running, else (<Z_v> array, info dict)."""
        return self._take(lib().tn_server_poll_ex, ticket)

    def wait(self, ticket, timeout=600.0):
        """(<Z_v>, info) once the job ends; None if it has not ended after
        `timeout` seconds (None: wait without a limit)."""
        if timeout is None:
            while True:
                r = self._take(lib().tn_server_wait_ex, ticket, C.c_double(3600.0))
                if r is not None:
                    return r
        return self._take(lib().tn_server_wait_ex, ticket, C.c_double(timeout))

    def stats(self):
        s = tn_server_stats()
        _check(lib().tn_server_get_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in tn_server_stats._fields_}

    def close(self):
        if self._h:
            lib().tn_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def chi_extrapolate(chis, values):
    """Least-squares fit values[i, k] = A_k + B_k / chis[i] (tn_chi_extrapolate).

    values: [len(chis), n_obs] (or [len(chis)]).  Returns (A, B, rms), A the
    chi -> infinity estimate of each observable."""
    x = np.ascontiguousarray(chis, dtype=np.float64).reshape(-1)
    v = np.ascontiguousarray(values, dtype=np.float64).reshape(len(x), -1)
    k = v.shape[1]
    a, b, r = np.zeros(k), np.zeros(k), np.zeros(k)
    P = C.POINTER(C.c_double)
    _check(lib().tn_chi_extrapolate(x.ctypes.data_as(P), v.ctypes.data_as(P), len(x), k,
                                    a.ctypes.data_as(P), b.ctypes.data_as(P),
                                    r.ctypes.data_as(P)))
    return a, b, r


def theta_chi_sweep(server, n, edges, colours, thetas, chis, steps, prec="tf32", **cfg):
    """A theta_h grid x chi ladder run as jobs of one server (they overlap on the
    device as the server admits them), then extrapolated linearly in 1/chi.

    Returns {"z": [n_theta, n_chi, n] <Z_v> after `steps` steps, "z_inf":
    [n_theta, n] the intercepts, "slope", "rms", "steps_done": [n_theta, n_chi]}."""
    tickets = {}
    for i, th in enumerate(thetas):
        for j, chi in enumerate(chis):
            tickets[(i, j)] = server.submit(n, edges, colours, int(chi), float(th), int(steps),
                                            prec=prec, **cfg)
    z = np.zeros((len(thetas), len(chis), n))
    done = np.zeros((len(thetas), len(chis)), dtype=np.int64)
    for (i, j), t in tickets.items():
        r = server.wait(t)
        if r is None:
            raise TNError(-7, "job %d did not finish in time" % t)
        z[i, j], info = r
        done[i, j] = info["steps_done"]
    fits = [chi_extrapolate(chis, z[i]) for i in range(len(thetas))]
    return {"z": z, "z_inf": np.stack([f[0] for f in fits]),
            "slope": np.stack([f[1] for f in fits]), "rms": np.stack([f[2] for f in fits]),
            "steps_done": done}


def selftest_bounded_wait(stream=None):
    """Flag word of the bounded-wait self-test (2: the wait timed out as it must)."""
    f = C.c_int32()
    _check(lib().tn_selftest_bounded_wait(C.c_void_p(stream), C.byref(f)))
    return f.value


def version():
    return lib().tn_version().decode()
