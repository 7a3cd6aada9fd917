"""Python binding of the C ABI in include/fdlb.h (argument marshalling only).

Every computation runs in libfdlb_gb300.so: the set-up on the host in C++, every step of the
solver in the CUDA kernels.  There is no fallback: if the library is missing or no GPU is
usable, calls raise.  PyTorch, when importable with CUDA, supplies the device workspace and
the stream; otherwise the library allocates its own device memory.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_int64, c_size_t, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfdlb_gb300.so")

CYL, SPH, CYL_Z = 0, 1, 2  # CYL_Z: the cylinder with p_z integrated out (the pair phi, chi)
FP64, FP32 = 0, 1
CHI_RET_FM, CHI_SET_LOCAL = 0, 1
QUAD_FULL, QUAD_HALF = 0, 1
NMOM = 9
MOMENT_NAMES = ("n", "u1", "u2", "u3", "T", "q1", "q2", "q3", "P12")

ERRORS = {0: "ok", 1: "EINVAL", 2: "ECUDA", 3: "ENOMEM", 4: "ENOTCONVERGED", 5: "ETIMEOUT", 6: "ENAN",
          7: "EIO", 8: "ENOGPU"}


class FdlbError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({code})")


class Params(ctypes.Structure):
    _fields_ = [
        ("geometry", c_int),
        ("R_in", c_double), ("R_out", c_double),
        ("n_cells", c_int),
        ("stretch_beta", c_double),
        ("Q_R", c_int), ("Q_2", c_int), ("Q_3", c_int),
        ("N_R", c_int), ("N_2", c_int), ("N_3", c_int),
        ("eta0", c_double), ("Kn", c_double), ("sigma", c_double),
        ("chi_model", c_int), ("precision", c_int),
        ("dt", c_double), ("cfl", c_double),
        ("T_wall", c_double * 2), ("u_wall", c_double * 2),
    ]


class Info(ctypes.Structure):
    _fields_ = [("C", c_double), ("sigma", c_double), ("n0", c_double), ("dt", c_double),
                ("R_first", c_double), ("R_last", c_double), ("n_cells", c_int), ("n_momenta", c_int),
                ("fm_band", c_int), ("precision", c_int), ("step", c_int64)]


_lib = None
_DP = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_FP = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")


def load_library():
    """Load the in-tree library (built by paper_2403_15051_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2403_15051_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    H = c_void_p
    sig = {
        "fdlb_create": (c_int, [POINTER(Params), c_void_p, POINTER(H)]),
        "fdlb_batch_create": (c_int, [POINTER(Params), c_int, c_void_p, POINTER(H)]),
        "fdlb_workspace_bytes": (c_int, [POINTER(Params), c_int, POINTER(c_size_t)]),
        "fdlb_create_in": (c_int, [POINTER(Params), c_int, c_void_p, c_void_p, c_size_t, POINTER(H)]),
        "fdlb_destroy": (None, [H]),
        "fdlb_set_wall": (c_int, [H, c_int, c_int, c_double, c_double]),
        "fdlb_init_uniform": (c_int, [H, c_int, c_double, c_double]),
        "fdlb_init_from_moments": (c_int, [H, c_int, _DP, _DP, _DP, _DP, c_int]),
        "fdlb_set_f": (c_int, [H, c_int, _DP]),
        "fdlb_get_f": (c_int, [H, c_int, _DP]),
        "fdlb_step": (c_int, [H, c_int64]),
        "fdlb_run_to_steady": (c_int, [H, c_double, c_int64, c_double, c_int, POINTER(c_int64), POINTER(c_double)]),
        "fdlb_run_to_steady_mixed": (c_int, [H, c_double, c_int64, c_double, c_int, c_void_p, c_size_t,
                                             POINTER(c_int64), POINTER(c_int64), POINTER(c_double)]),
        "fdlb_polish_workspace_bytes": (c_int, [H, POINTER(c_size_t)]),
        "fdlb_eval_rhs": (c_int, [H, c_int, _DP]),
        "fdlb_get_moments": (c_int, [H, c_int, c_void_p, c_int]),
        "fdlb_get_closure": (c_int, [H, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
        "fdlb_get_diagnostics": (c_int, [H, c_int, POINTER(c_double), POINTER(c_double), POINTER(c_int64)]),
        "fdlb_get_info": (c_int, [H, c_int, POINTER(Info)]),
        "fdlb_save": (c_int, [H, ctypes.c_char_p]),
        "fdlb_load": (c_int, [H, ctypes.c_char_p]),
        "fdlb_error_string": (ctypes.c_char_p, [c_int]),
        "fdlb_set_tiling": (c_int, [H, c_int, c_int, c_int]),
        "fdlb_set_closure_cells": (c_int, [H, c_int]),
        "fdlb_set_closure_form": (c_int, [H, c_int, POINTER(c_int)]),
        "fdlb_set_stall_checks": (c_int, [H, c_int]),
        "fdlb_step_change": (c_int, [H, POINTER(c_double)]),
        "fdlb_get_stage_kernel": (c_int, [H, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
        "fdlb_set_stage_min_blocks": (c_int, [H, c_int, POINTER(c_int)]),
        "fdlb_set_programmatic_launch": (c_int, [H, c_int]),
        "fdlb_set_tensor_contraction": (c_int, [H, c_int, POINTER(c_int)]),
        "fdlb_set_persistent_step": (c_int, [H, c_int, POINTER(c_int)]),
        "fdlb_set_wait_test": (c_int, [H, c_int, c_int]),
        "fdlb_clear_error": (c_int, [H]),
        "fdlb_step_kernel_times": (c_int, [H, POINTER(c_double), POINTER(c_int64), POINTER(c_int64)]),
        "fdlb_autotune": (c_int, [H, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
        "fdlb_set_autotune": (c_int, [H, c_int]),
        "fdlb_get_tiling": (c_int, [H, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
        "fdlb_launch_count": (c_int64, [H]),
        "fdlb_set_graph_steps": (c_int, [H, c_int]),
        "fdlb_set_kernel_timing": (c_int, [H, c_int]),
        "fdlb_kernel_times": (c_int, [H, POINTER(c_double), POINTER(c_int64), POINTER(c_double), POINTER(c_int64)]),
        "fdlb_get_stream": (c_int, [H, POINTER(c_void_p)]),
        "fdlb_set_state_raw": (c_int, [H, c_int, c_void_p, c_int]),
        "fdlb_get_state_raw": (c_int, [H, c_int, c_void_p, c_int]),
        "fdlb_state_bytes": (c_int, [H, POINTER(c_size_t)]),
        "fdlb_moments_noalloc": (c_int, [c_int, c_int, c_int, c_int, _DP, c_int, c_void_p, c_void_p, c_void_p]),
        "fdlb_fp32_fma_peak": (c_int, [c_void_p, c_int, POINTER(c_double), POINTER(c_double)]),
        "fdlb_nn_create": (c_int, [c_int, c_int, c_int, c_int, c_int, c_int, c_void_p, POINTER(H)]),
        "fdlb_nn_destroy": (None, [H]),
        "fdlb_nn_num_params": (c_int, [H, POINTER(c_int64)]),
        "fdlb_nn_set_params": (c_int, [H, _FP]),
        "fdlb_nn_get_params": (c_int, [H, _FP]),
        "fdlb_nn_init_params": (c_int, [H, ctypes.c_uint64]),
        "fdlb_nn_forward": (c_int, [H, _FP, c_int, _FP]),
        "fdlb_nn_loss_grad": (c_int, [H, _FP, _FP, c_int, POINTER(ctypes.c_float), c_void_p]),
        "fdlb_nn_train_step": (c_int, [H, _FP, _FP, c_int, ctypes.c_float, POINTER(ctypes.c_float)]),
        "fdlb_nn_warm_start": (c_int, [H, H, c_int, _FP]),
        "fdlb_quadrature": (c_int, [c_int, c_int, _DP, _DP]),
        "fdlb_derivative_matrix": (c_int, [c_int, c_int, _DP]),
        "fdlb_physical_parameters": (c_int, [c_double, c_double, c_double, POINTER(c_double), POINTER(c_double),
                                             POINTER(c_double)]),
        "fdlb_grid": (c_int, [c_int, c_double, c_double, c_double, c_int, c_double, c_void_p, c_void_p, c_void_p,
                              c_void_p]),
        "fdlb_fm_weights": (c_int, [c_int, c_double, c_double, c_double, c_int, c_double, _DP]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc, where):
    if rc != 0:
        raise FdlbError(rc, where)


def _precision_code(prec) -> int:
    if prec not in ("fp32", "fp64", FP32, FP64):
        raise ValueError(f"precision must be 'fp32' or 'fp64', not {prec!r}")
    return FP32 if prec in ("fp32", FP32) else FP64


def make_params(d: dict) -> Params:
    """fdlb_params from a workload dictionary (see workloads.py)."""
    p = Params()
    p.geometry = int(d.get("geometry", CYL))
    p.R_in, p.R_out = float(d["R_in"]), float(d["R_out"])
    p.n_cells = int(d["n_cells"])
    p.stretch_beta = float(d.get("beta", 0.0) or 0.0)
    p.Q_R, p.Q_2, p.Q_3 = int(d["Q_R"]), int(d["Q_2"]), int(d["Q_3"])
    p.N_R, p.N_2, p.N_3 = (int(d.get(k, -1)) if d.get(k) is not None else -1 for k in ("N_R", "N_2", "N_3"))
    p.eta0 = float(d["eta0"])
    p.Kn = float(d.get("Kn") or 0.0)
    p.sigma = float(d.get("sigma") or 0.0)
    p.chi_model = int(d.get("chi_model", CHI_RET_FM))
    p.precision = _precision_code(d.get("precision", "fp64"))
    p.dt = float(d.get("dt") or 0.0)
    p.cfl = float(d.get("cfl") or 0.0)
    T = d.get("T_wall", (1.0, 1.0))
    u = d.get("u_wall", (0.0, 0.0))
    p.T_wall[0], p.T_wall[1] = float(T[0]), float(T[1])
    p.u_wall[0], p.u_wall[1] = float(u[0]), float(u[1])
    return p


def _torch_cuda():
    try:
        import torch
    except Exception:
        return None
    return torch if torch.cuda.is_available() else None


class Solver:
    """One handle of the library: a single instance or a batch of instances."""

    def __init__(self, params, stream=None, use_torch_workspace=True):
        L = load_library()
        if isinstance(params, dict):
            params = [params]
        self.param_dicts = list(params)
        n = len(params)
        arr = (Params * n)(*[make_params(d) for d in params])
        self._arr = arr
        self.n_instances = n
        torch = _torch_cuda() if use_torch_workspace else None
        if stream is None and torch is not None:
            stream = torch.cuda.current_stream().cuda_stream
        self._stream = c_void_p(int(stream) if stream is not None else 0)
        self._workspace = None
        h = c_void_p()
        if torch is not None:
            nb = c_size_t()
            _check(L.fdlb_workspace_bytes(arr, n, byref(nb)), "fdlb_workspace_bytes")
            self._workspace = torch.empty(int(nb.value) + 256, dtype=torch.uint8, device="cuda")
            base = self._workspace.data_ptr()
            aligned = (base + 255) // 256 * 256
            _check(L.fdlb_create_in(arr, n, self._stream, c_void_p(aligned), c_size_t(nb.value), byref(h)),
                   "fdlb_create_in")
        else:
            _check(L.fdlb_batch_create(arr, n, self._stream, byref(h)), "fdlb_batch_create")
        self._h = h
        self._L = L
        self.infos = [self.info(q) for q in range(n)]

    # ------------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "_h", None):
            self._L.fdlb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ helpers
    def shape(self, q=0):
        d = self.param_dicts[q]
        n3 = 2 if int(d.get("geometry", CYL)) == CYL_Z else int(d["Q_3"])  # the reduced pair (phi, chi)
        return (int(d["n_cells"]), 2 * int(d["Q_R"]), int(d["Q_2"]), n3)

    def info(self, q=0) -> dict:
        inf = Info()
        _check(self._L.fdlb_get_info(self._h, q, byref(inf)), "fdlb_get_info")
        return {k: getattr(inf, k) for k, _ in Info._fields_}

    # ------------------------------------------------------------------ set-up
    def set_wall(self, q, side, T_w, u_t=0.0):
        _check(self._L.fdlb_set_wall(self._h, q, side, T_w, u_t), "fdlb_set_wall")

    def init_uniform(self, q=-1, n0=0.0, T0=0.0):
        _check(self._L.fdlb_init_uniform(self._h, q, n0, T0), "fdlb_init_uniform")

    def init_from_moments(self, q, n, u2, T, qR):
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (n, u2, T, qR)]
        _check(self._L.fdlb_init_from_moments(self._h, q, *a, len(a[0])), "fdlb_init_from_moments")

    def set_f(self, f, q=0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.shape != self.shape(q):
            raise ValueError(f"f must have shape {self.shape(q)}")
        _check(self._L.fdlb_set_f(self._h, q, f.reshape(-1)), "fdlb_set_f")

    def get_f(self, q=0):
        out = np.empty(self.shape(q))
        _check(self._L.fdlb_get_f(self._h, q, out.reshape(-1)), "fdlb_get_f")
        return out

    # ------------------------------------------------------------------ stepping
    def step(self, n=1):
        _check(self._L.fdlb_step(self._h, int(n)), "fdlb_step")

    def run_to_steady(self, tol=1e-8, max_steps=1_000_000, max_seconds=0.0, check_every=100):
        n = self.n_instances
        st = (c_int64 * n)()
        res = (c_double * n)()
        rc = self._L.fdlb_run_to_steady(self._h, tol, int(max_steps), float(max_seconds), int(check_every), st, res)
        return rc, np.array(st[:], dtype=np.int64), np.array(res[:])

    def run_to_steady_mixed(self, tol=1e-8, max_steps=1_000_000, max_seconds=0.0, check_every=100):
        """FP32 to the tolerance, then the library's FP64 polish (fdlb_run_to_steady_mixed); the
        FP64 copy's device memory comes from torch when this handle's does.  Returns (status,
        FP32 steps, FP64 steps, residuals)."""
        n = self.n_instances
        s32, s64 = (c_int64 * n)(), (c_int64 * n)()
        res = (c_double * n)()
        ws, nb_v = None, 0
        torch = _torch_cuda() if self._workspace is not None else None
        if torch is not None:
            nb = c_size_t()
            _check(self._L.fdlb_polish_workspace_bytes(self._h, byref(nb)), "fdlb_polish_workspace_bytes")
            nb_v = int(nb.value)
            ws = torch.empty(nb_v + 256, dtype=torch.uint8, device="cuda")
        ptr = c_void_p((ws.data_ptr() + 255) // 256 * 256 if ws is not None else 0)
        rc = self._L.fdlb_run_to_steady_mixed(self._h, tol, int(max_steps), float(max_seconds), int(check_every), ptr,
                                              c_size_t(nb_v), s32, s64, res)
        del ws
        return rc, np.array(s32[:], dtype=np.int64), np.array(s64[:], dtype=np.int64), np.array(res[:])

    def eval_rhs(self, q=0):
        out = np.empty(self.shape(q))
        _check(self._L.fdlb_eval_rhs(self._h, q, out.reshape(-1)), "fdlb_eval_rhs")
        return out

    # ------------------------------------------------------------------ outputs
    def moments(self, q=0) -> dict:
        N = self.shape(q)[0]
        out = np.empty((N, NMOM))
        _check(self._L.fdlb_get_moments(self._h, q, out.ctypes.data_as(c_void_p), 0), "fdlb_get_moments")
        return {k: out[:, i].copy() for i, k in enumerate(MOMENT_NAMES)}

    def moments_device(self, q, out_ptr):
        _check(self._L.fdlb_get_moments(self._h, q, c_void_p(out_ptr), 1), "fdlb_get_moments")

    def closure(self, q=0) -> dict:
        N = self.shape(q)[0]
        nbar, chi, tau, nw = np.empty(N), np.empty(N), np.empty(N), np.empty(2)
        _check(self._L.fdlb_get_closure(self._h, q, nbar.ctypes.data_as(c_void_p), chi.ctypes.data_as(c_void_p),
                                        tau.ctypes.data_as(c_void_p), nw.ctypes.data_as(c_void_p)),
               "fdlb_get_closure")
        return {"nbar": nbar, "chi": chi, "tau": tau, "n_wall": nw}

    def diagnostics(self, q=0):
        m, r, s = c_double(), c_double(), c_int64()
        rc = self._L.fdlb_get_diagnostics(self._h, q, byref(m), byref(r), byref(s))
        return rc, m.value, r.value, s.value

    def save(self, path):
        _check(self._L.fdlb_save(self._h, path.encode()), "fdlb_save")

    def load(self, path):
        _check(self._L.fdlb_load(self._h, path.encode()), "fdlb_load")

    def set_tiling(self, cells=0, slice_k=0, threads=0):
        _check(self._L.fdlb_set_tiling(self._h, cells, slice_k, threads), "fdlb_set_tiling")

    def set_tensor_contraction(self, enable):
        used = c_int()
        _check(self._L.fdlb_set_tensor_contraction(self._h, 1 if enable else 0, byref(used)),
               "fdlb_set_tensor_contraction")
        return bool(used.value)

    def set_persistent_step(self, enable):
        """Whole steps in one persistent launch (default off); returns whether it applies to
        this handle.  enable=None only reports."""
        used = c_int()
        flag = -1 if enable is None else (1 if enable else 0)
        _check(self._L.fdlb_set_persistent_step(self._h, flag, byref(used)), "fdlb_set_persistent_step")
        return bool(used.value)

    def set_wait_test(self, tx_extra_bytes=0, barrier_extra=0):
        """Test hooks that make the bounded device waits run out (0, 0 in use)."""
        _check(self._L.fdlb_set_wait_test(self._h, tx_extra_bytes, barrier_extra), "fdlb_set_wait_test")

    def clear_error(self):
        _check(self._L.fdlb_clear_error(self._h), "fdlb_clear_error")

    def set_programmatic_launch(self, enable):
        _check(self._L.fdlb_set_programmatic_launch(self._h, 1 if enable else 0), "fdlb_set_programmatic_launch")

    def set_closure_cells(self, cells):
        _check(self._L.fdlb_set_closure_cells(self._h, cells), "fdlb_set_closure_cells")

    def step_change(self):
        """One step; per instance the relative L2 change ||f^{n+1} - f^n|| / ||f^n|| (FP64 sums)."""
        out = (c_double * self.n_instances)()
        _check(self._L.fdlb_step_change(self._h, out), "fdlb_step_change")
        return np.array(out[:])

    def set_stall_checks(self, checks):
        """Instances whose residual has not halved its best value for `checks` consecutive checks
        stop stepping in run_to_steady (0: never)."""
        _check(self._L.fdlb_set_stall_checks(self._h, int(checks)), "fdlb_set_stall_checks")

    def closure_form(self, form=-1):
        """0: the chain form, 1: the batch form, -1: no change; returns the form in use."""
        u = c_int()
        _check(self._L.fdlb_set_closure_form(self._h, int(form), byref(u)), "fdlb_set_closure_form")
        return u.value

    def stage_min_blocks(self, min_blocks=-1):
        """Pins the stage kernel's register bound (1, or 2, 3, 5 where built; -1: no change);
        returns the bound in use (fdlb_set_stage_min_blocks in include/fdlb.h)."""
        u = c_int()
        _check(self._L.fdlb_set_stage_min_blocks(self._h, int(min_blocks), byref(u)), "fdlb_set_stage_min_blocks")
        return u.value

    def autotune(self):
        b, k, t = c_int(), c_int(), c_int()
        _check(self._L.fdlb_autotune(self._h, byref(b), byref(k), byref(t)), "fdlb_autotune")
        return b.value, k.value, t.value

    def set_autotune(self, mode):
        """0 off, 1 tune batches at their first step (default), 2 tune every handle."""
        _check(self._L.fdlb_set_autotune(self._h, int(mode)), "fdlb_set_autotune")

    def tiling(self) -> dict:
        b, k, t, c = c_int(), c_int(), c_int(), c_int()
        _check(self._L.fdlb_get_tiling(self._h, byref(b), byref(k), byref(t), byref(c)), "fdlb_get_tiling")
        form = self.closure_form()
        vw, nv, mb = c_int(), c_int(), c_int()
        _check(self._L.fdlb_get_stage_kernel(self._h, byref(vw), byref(nv), byref(mb)), "fdlb_get_stage_kernel")
        return {"cells_per_tile": b.value, "slice_k": k.value, "threads": t.value,
                "closure_cells": 28 if form == 1 else c.value, "closure_form": "batch" if form == 1 else "chain",
                "stage_vector_width": vw.value, "stage_vectors_per_thread": nv.value,
                "stage_min_blocks_per_sm": mb.value}

    def launch_count(self):
        return int(self._L.fdlb_launch_count(self._h))

    def set_graph_steps(self, steps):
        _check(self._L.fdlb_set_graph_steps(self._h, int(steps)), "fdlb_set_graph_steps")

    def set_kernel_timing(self, on=True):
        _check(self._L.fdlb_set_kernel_timing(self._h, 1 if on else 0), "fdlb_set_kernel_timing")

    def kernel_times(self):
        """(stream-kernel ms, launches, closure-kernel ms, launches) accumulated since the last call."""
        sm, ns, cm, nc = c_double(), c_int64(), c_double(), c_int64()
        _check(self._L.fdlb_kernel_times(self._h, byref(sm), byref(ns), byref(cm), byref(nc)), "fdlb_kernel_times")
        return sm.value, ns.value, cm.value, nc.value

    def step_kernel_times(self):
        """(persistent step-kernel ms, launches, steps) accumulated since the last call."""
        ms, nl, ns = c_double(), c_int64(), c_int64()
        _check(self._L.fdlb_step_kernel_times(self._h, byref(ms), byref(nl), byref(ns)), "fdlb_step_kernel_times")
        return ms.value, nl.value, ns.value

    def stream_handle(self):
        s = c_void_p()
        _check(self._L.fdlb_get_stream(self._h, byref(s)), "fdlb_get_stream")
        return int(s.value or 0)

    def set_state_raw(self, ptr, q=0, on_device=False):
        _check(self._L.fdlb_set_state_raw(self._h, q, c_void_p(ptr), 1 if on_device else 0), "fdlb_set_state_raw")

    def get_state_raw(self, ptr, q=0, on_device=False):
        _check(self._L.fdlb_get_state_raw(self._h, q, c_void_p(ptr), 1 if on_device else 0), "fdlb_get_state_raw")

    def raw_elements(self, q=0):
        n = self.shape(q)
        return n[0] * n[1] * n[2] * n[3]

    def state_bytes(self):
        """Bytes of the whole batch's populations as the library stores them (instance -1 of
        set_state_raw / get_state_raw)."""
        nb = c_size_t()
        _check(self._L.fdlb_state_bytes(self._h, byref(nb)), "fdlb_state_bytes")
        return int(nb.value)

    def moments_all(self, out=None) -> np.ndarray:
        """Moments of every instance, [total cells][NMOM] in instance order.  `out`: an FP64 host
        array of that shape to fill (page-locked memory copies at the full link rate)."""
        N = sum(self.shape(q)[0] for q in range(self.n_instances))
        if out is None:
            out = np.empty((N, NMOM))
        if out.shape != (N, NMOM) or out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a C-contiguous float64 array of shape (%d, %d)" % (N, NMOM))
        _check(self._L.fdlb_get_moments(self._h, -1, out.ctypes.data_as(c_void_p), 0), "fdlb_get_moments")
        return out


# ---------------------------------------------------------------------- host-only set-up
def quadrature(kind, Q):
    L = load_library()
    n = 2 * Q if kind == QUAD_HALF else Q
    x, w = np.empty(n), np.empty(n)
    _check(L.fdlb_quadrature(kind, Q, x, w), "fdlb_quadrature")
    return x, w


def moments_noalloc(precision, Q_R, Q_2, Q_3, n_cells, f_dev_ptr, moments_dev_ptr, stream=0):
    """Per-cell moments of device populations in the library layout, without any device
    allocation by the library (see fdlb_moments_noalloc in include/fdlb.h)."""
    L = load_library()
    nodes = np.concatenate([quadrature(QUAD_HALF, Q_R)[0], quadrature(QUAD_FULL, Q_2)[0],
                            quadrature(QUAD_FULL, Q_3)[0]])
    prec = _precision_code(precision)
    _check(L.fdlb_moments_noalloc(prec, Q_R, Q_2, Q_3, nodes, int(n_cells), c_void_p(f_dev_ptr),
                                  c_void_p(moments_dev_ptr), c_void_p(int(stream))), "fdlb_moments_noalloc")


def fp32_fma_peak(stream=0, repeats=5):
    """Measured FP32 FMA rate of the current device in TFLOP/s and the timed launch's duration in
    ms (fdlb_fp32_fma_peak in include/fdlb.h)."""
    L = load_library()
    tf, ms = c_double(), c_double()
    _check(L.fdlb_fp32_fma_peak(c_void_p(int(stream)), int(repeats), byref(tf), byref(ms)), "fdlb_fp32_fma_peak")
    return tf.value, ms.value


def derivative_matrix(kind, Q):
    L = load_library()
    n = 2 * Q if kind == QUAD_HALF else Q
    K = np.empty((n, n))
    _check(L.fdlb_derivative_matrix(kind, Q, K.reshape(-1)), "fdlb_derivative_matrix")
    return K


def physical_parameters(Kn, eta0, L_gap):
    L = load_library()
    C, s, n0 = c_double(), c_double(), c_double()
    _check(L.fdlb_physical_parameters(Kn, eta0, L_gap, byref(C), byref(s), byref(n0)), "fdlb_physical_parameters")
    return C.value, s.value, n0.value


def grid(geometry, R_in, R_out, sigma, n_cells, beta=0.0):
    L = load_library()
    Rc, Rf, V, k = np.empty(n_cells), np.empty(n_cells + 1), np.empty(n_cells), np.empty(n_cells)
    _check(L.fdlb_grid(geometry, R_in, R_out, sigma, n_cells, beta, *(a.ctypes.data_as(c_void_p) for a in (Rc, Rf, V, k))),
           "fdlb_grid")
    return Rc, Rf, V, k


def fm_weights(geometry, R_in, R_out, sigma, n_cells, beta=0.0):
    L = load_library()
    W = np.empty((n_cells, n_cells))
    _check(L.fdlb_fm_weights(geometry, R_in, R_out, sigma, n_cells, beta, W.reshape(-1)), "fdlb_fm_weights")
    return W


class WarmStartNet:
    """The learned warm-start network of the library (fdlb_nn_* in include/fdlb.h)."""

    def __init__(self, width=64, modes=6, layers=4, hidden=128, n_points=256, max_batch=64, stream=None):
        L = load_library()
        h = c_void_p()
        _check(L.fdlb_nn_create(width, modes, layers, hidden, n_points, max_batch,
                                c_void_p(int(stream) if stream else 0), byref(h)), "fdlb_nn_create")
        self._h, self._L = h, L
        self.n_points, self.max_batch = n_points, max_batch
        cnt = c_int64()
        _check(L.fdlb_nn_num_params(h, byref(cnt)), "fdlb_nn_num_params")
        self.n_params = int(cnt.value)

    def close(self):
        if getattr(self, "_h", None):
            self._L.fdlb_nn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        assert t.size == self.n_params
        _check(self._L.fdlb_nn_set_params(self._h, t), "fdlb_nn_set_params")

    def init_params(self, seed=0):
        _check(self._L.fdlb_nn_init_params(self._h, int(seed)), "fdlb_nn_init_params")

    def get_params(self):
        t = np.empty(self.n_params, np.float32)
        _check(self._L.fdlb_nn_get_params(self._h, t), "fdlb_nn_get_params")
        return t

    def forward(self, raw):
        raw = np.ascontiguousarray(raw, dtype=np.float32).reshape(-1, 5)
        out = np.empty((raw.shape[0], self.n_points, 4), np.float32)
        _check(self._L.fdlb_nn_forward(self._h, raw, raw.shape[0], out), "fdlb_nn_forward")
        return out

    def loss_grad(self, raw, target):
        raw = np.ascontiguousarray(raw, dtype=np.float32).reshape(-1, 5)
        target = np.ascontiguousarray(target, dtype=np.float32)
        loss = ctypes.c_float()
        g = np.empty(self.n_params, np.float32)
        _check(self._L.fdlb_nn_loss_grad(self._h, raw, target, raw.shape[0], byref(loss), g.ctypes.data_as(c_void_p)),
               "fdlb_nn_loss_grad")
        return float(loss.value), g

    def train_step(self, raw, target, lr):
        raw = np.ascontiguousarray(raw, dtype=np.float32).reshape(-1, 5)
        target = np.ascontiguousarray(target, dtype=np.float32)
        loss = ctypes.c_float()
        _check(self._L.fdlb_nn_train_step(self._h, raw, target, raw.shape[0], float(lr), byref(loss)),
               "fdlb_nn_train_step")
        return float(loss.value)

    def warm_start(self, solver, instance, raw):
        raw = np.ascontiguousarray(raw, dtype=np.float32).reshape(5)
        _check(self._L.fdlb_nn_warm_start(self._h, solver._h, instance, raw), "fdlb_nn_warm_start")
