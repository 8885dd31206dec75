"""Python binding of the C-ABI in include/esp.h (argument marshalling only).

Every function has the name of its C entry point. Arrays may be NumPy arrays
(host memory, ``where=ESP_HOST``) or torch tensors (``where`` follows the
tensor's device). All computation runs in libesp_gb300.so; this module never
computes anything itself and raises if the library is not built.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

ESP_OK = 0
ESP_KERNEL_PSWF, ESP_KERNEL_GAUSS = 0, 1
ESP_WINDOW_PSWF, ESP_WINDOW_BSPLINE = 0, 1
ESP_DIFF_AD, ESP_DIFF_IK = 0, 1
ESP_FP32, ESP_FP64 = 0, 1
ESP_HOST, ESP_DEVICE = 0, 1

STATUS = {
    0: "ESP_OK", 1: "ESP_ERR_INVALID_ARG", 2: "ESP_ERR_CUTOFF_TOO_LARGE", 3: "ESP_ERR_NOT_NEUTRAL",
    4: "ESP_ERR_NONFINITE", 5: "ESP_ERR_OOM", 6: "ESP_ERR_CUDA", 7: "ESP_ERR_CUFFT",
    8: "ESP_ERR_TIMEOUT", 9: "ESP_ERR_BUSY", 10: "ESP_ERR_UNSUPPORTED", 11: "ESP_ERR_INTERNAL",
    12: "ESP_ERR_NOT_READY",
}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libesp_gb300.so")


class EspError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class esp_box(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double * 3)]


class esp_cell(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double * 3), ("b", ctypes.c_double * 3), ("c", ctypes.c_double * 3)]


class esp_plan_opts(ctypes.Structure):
    _fields_ = [
        ("r_c", ctypes.c_double), ("P", ctypes.c_int), ("n_f", ctypes.c_int),
        ("c", ctypes.c_double), ("c1", ctypes.c_double), ("alpha", ctypes.c_double),
        ("kernel", ctypes.c_int), ("precision", ctypes.c_int), ("prefactor", ctypes.c_double),
        ("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("allow_background", ctypes.c_int),
        ("brick_cells", ctypes.c_int), ("timeout_ms", ctypes.c_double),
        ("cell_reach", ctypes.c_int), ("window", ctypes.c_int), ("near_variant", ctypes.c_int),
        ("diff", ctypes.c_int), ("virial", ctypes.c_int), ("reserved", ctypes.c_int * 3),
    ]


class esp_plan_params(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double), ("r_c", ctypes.c_double), ("h", ctypes.c_double),
        ("c", ctypes.c_double), ("c1", ctypes.c_double), ("alpha", ctypes.c_double),
        ("prefactor", ctypes.c_double), ("alias_estimate", ctypes.c_double),
        ("si_fit_error", ctypes.c_double), ("near_fit_error", ctypes.c_double),
        ("N", ctypes.c_int64), ("P", ctypes.c_int), ("n_f", ctypes.c_int),
        ("kernel", ctypes.c_int), ("precision", ctypes.c_int), ("n_cells", ctypes.c_int),
        ("cell_reach", ctypes.c_int), ("near_terms", ctypes.c_int),
        ("brick_cells", ctypes.c_int), ("tile", ctypes.c_int), ("si_degree", ctypes.c_int),
        ("near_degree", ctypes.c_int), ("device_bytes", ctypes.c_size_t), ("window", ctypes.c_int),
        ("diff", ctypes.c_int), ("virial", ctypes.c_int), ("triclinic", ctypes.c_int),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class esp_md_params(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double), ("k_bond", ctypes.c_double), ("r0", ctypes.c_double),
        ("k_angle", ctypes.c_double), ("theta0", ctypes.c_double), ("lj_sigma", ctypes.c_double),
        ("lj_epsilon", ctypes.c_double), ("lj_cutoff", ctypes.c_double), ("mass_O", ctypes.c_double),
        ("mass_H", ctypes.c_double), ("reserved", ctypes.c_int * 8),
    ]


class esp_server_opts(ctypes.Structure):
    _fields_ = [
        ("memory_budget", ctypes.c_size_t), ("device", ctypes.c_int), ("max_inflight", ctypes.c_int),
        ("r_c", ctypes.c_double), ("precision", ctypes.c_int), ("kernel", ctypes.c_int),
        ("timeout_ms", ctypes.c_double), ("reserved", ctypes.c_int * 8),
    ]


class esp_server_counters(ctypes.Structure):
    _fields_ = [
        ("completed", ctypes.c_int64), ("failed", ctypes.c_int64), ("pending", ctypes.c_int64),
        ("running", ctypes.c_int64), ("atoms_done", ctypes.c_double), ("plans_resident", ctypes.c_int64),
        ("plans_created", ctypes.c_int64), ("evictions", ctypes.c_int64), ("device_bytes", ctypes.c_size_t),
        ("memory_budget", ctypes.c_size_t), ("latency_p50_ms", ctypes.c_double),
        ("latency_p99_ms", ctypes.c_double), ("latency_max_ms", ctypes.c_double), ("wall_ms", ctypes.c_double),
        ("peak_inflight", ctypes.c_int64), ("peak_concurrent", ctypes.c_int64), ("overlap_ms", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_SIGNATURES = {
    "esp_plan_opts_init": (None, [ctypes.POINTER(esp_plan_opts)]),
    "esp_plan": (ctypes.c_int, [ctypes.POINTER(esp_box), ctypes.c_int64, ctypes.c_double,
                                ctypes.POINTER(esp_plan_opts), ctypes.POINTER(_P)]),
    "esp_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(esp_plan_params)]),
    "esp_set_exclusions": (ctypes.c_int, [_P, _P, ctypes.c_int64]),
    "esp_md_params_init": (None, [ctypes.POINTER(esp_md_params)]),
    "esp_md_create": (ctypes.c_int, [_P, ctypes.POINTER(esp_md_params), _P, _P, ctypes.POINTER(_P)]),
    "esp_md_run": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "esp_md_state": (ctypes.c_int, [_P, _P, _P]),
    "esp_md_destroy": (ctypes.c_int, [_P]),
    "esp_plan_cell": (ctypes.c_int, [ctypes.POINTER(esp_cell), ctypes.c_int64, ctypes.c_double,
                                     ctypes.POINTER(esp_plan_opts), ctypes.POINTER(_P)]),
    "esp_plan_query_cell": (ctypes.c_int, [ctypes.POINTER(esp_cell), ctypes.c_int64, ctypes.c_double,
                                           ctypes.POINTER(esp_plan_opts), ctypes.POINTER(esp_plan_params)]),
    "esp_influence_query": (ctypes.c_int, [ctypes.POINTER(esp_box), ctypes.POINTER(esp_cell), ctypes.c_int64,
                                           ctypes.c_double, ctypes.POINTER(esp_plan_opts), _D,
                                           ctypes.POINTER(ctypes.c_int64)]),
    "esp_plan_query": (ctypes.c_int, [ctypes.POINTER(esp_box), ctypes.c_int64, ctypes.c_double,
                                      ctypes.POINTER(esp_plan_opts), ctypes.POINTER(esp_plan_params)]),
    "esp_set_charges": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "esp_set_charges_f32": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "esp_set_positions": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "esp_set_positions_f32": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "esp_compute": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int]),
    "esp_compute_f32": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int]),
    "esp_synchronize": (ctypes.c_int, [_P]),
    "esp_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "esp_phase_times": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
    "esp_last_spectral_energy": (ctypes.c_int, [_P, _D, _D]),
    "esp_last_virial": (ctypes.c_int, [_P, _D]),
    "esp_step": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int]),
    "esp_batch_last_virial": (ctypes.c_int, [_P, _D]),
    "esp_destroy": (ctypes.c_int, [_P]),
    "esp_batch_create": (ctypes.c_int, [ctypes.POINTER(esp_box), ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                        ctypes.c_double, ctypes.POINTER(esp_plan_opts), ctypes.POINTER(_P)]),
    "esp_batch_query": (ctypes.c_int, [ctypes.POINTER(esp_box), ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                       ctypes.c_double, ctypes.POINTER(esp_plan_opts),
                                       ctypes.POINTER(esp_plan_params)]),
    "esp_batch_info": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(esp_plan_params)]),
    "esp_batch_set_charges": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "esp_batch_compute": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int]),
    "esp_batch_synchronize": (ctypes.c_int, [_P]),
    "esp_batch_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "esp_batch_phase_times": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
    "esp_batch_destroy": (ctypes.c_int, [_P]),
    "esp_autotune": (ctypes.c_int, [ctypes.POINTER(esp_box), ctypes.c_int64, ctypes.c_double,
                                    ctypes.POINTER(esp_plan_opts), _P, _P, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(esp_plan_opts), _D]),
    "esp_server_opts_init": (None, [ctypes.POINTER(esp_server_opts)]),
    "esp_server_create": (ctypes.c_int, [ctypes.POINTER(esp_server_opts), ctypes.POINTER(_P)]),
    "esp_server_add_system": (ctypes.c_int, [_P, ctypes.POINTER(esp_box), ctypes.c_int64, _P,
                                             ctypes.POINTER(ctypes.c_int)]),
    "esp_server_submit": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, _P, ctypes.POINTER(ctypes.c_int64)]),
    "esp_server_poll": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]),
    "esp_server_wait": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, _P, _P, _P, _D]),
    "esp_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(esp_server_counters)]),
    "esp_server_reset_stats": (ctypes.c_int, [_P]),
    "esp_server_destroy": (ctypes.c_int, [_P]),
    "esp_local_part_static": (ctypes.c_int, [ctypes.POINTER(esp_box), ctypes.c_int64, ctypes.c_double,
                                             ctypes.POINTER(esp_plan_opts), _P, _P, _P, _P, _P]),
    "esp_last_error": (ctypes.c_char_p, []),
    "esp_version": (ctypes.c_char_p, []),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libesp_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != ESP_OK:
        msg = load_library().esp_last_error()
        raise EspError(status, msg.decode() if msg else "")


def _ptr(x, dtype=None):
    """(pointer, where) of a NumPy array or a torch tensor (None -> NULL)."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and x.dtype != dtype:
            raise TypeError(f"expected {dtype}, got {x.dtype}")
        return ctypes.c_void_p(x.ctypes.data), ESP_HOST
    # torch tensor (duck-typed to keep torch optional here)
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), (ESP_DEVICE if x.is_cuda else ESP_HOST)
    if isinstance(x, int):
        return ctypes.c_void_p(x), None
    raise TypeError(f"unsupported buffer type {type(x)}")


def esp_plan_opts_init() -> esp_plan_opts:
    o = esp_plan_opts()
    load_library().esp_plan_opts_init(ctypes.byref(o))
    return o


def make_opts(**kw) -> esp_plan_opts:
    o = esp_plan_opts_init()
    for k, v in kw.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = int(getattr(v, "cuda_stream", v))
        setattr(o, k, v)
    return o


def esp_plan(L: float, N: int, tolerance: float, opts: esp_plan_opts | None = None, **kw) -> int:
    if opts is None:
        opts = make_opts(**kw)
    box = esp_box((ctypes.c_double * 3)(L, L, L))
    out = _P()
    _check(load_library().esp_plan(ctypes.byref(box), int(N), float(tolerance), ctypes.byref(opts),
                                   ctypes.byref(out)))
    return out.value


def esp_plan_query(L: float, N: int, tolerance: float, opts: esp_plan_opts | None = None, **kw) -> dict:
    """Planner only (no GPU needed): the parameters esp_plan would choose."""
    if opts is None:
        opts = make_opts(**kw)
    box = esp_box((ctypes.c_double * 3)(L, L, L))
    p = esp_plan_params()
    _check(load_library().esp_plan_query(ctypes.byref(box), int(N), float(tolerance), ctypes.byref(opts),
                                         ctypes.byref(p)))
    return p.as_dict()


def _cell(H) -> esp_cell:
    """esp_cell from the 3x3 box matrix H whose columns are the cell vectors."""
    H = np.asarray(H, dtype=np.float64)
    if H.shape != (3, 3):
        raise ValueError("H must be 3x3 (columns a, b, c)")
    d3 = ctypes.c_double * 3
    return esp_cell(d3(*H[:, 0]), d3(*H[:, 1]), d3(*H[:, 2]))


def esp_plan_cell(H, N: int, tolerance: float, opts: esp_plan_opts | None = None, **kw) -> int:
    """Plan for a triclinic cell; H has the cell vectors a, b, c as columns."""
    if opts is None:
        opts = make_opts(**kw)
    cell = _cell(H)
    out = _P()
    _check(load_library().esp_plan_cell(ctypes.byref(cell), int(N), float(tolerance), ctypes.byref(opts),
                                        ctypes.byref(out)))
    return out.value


def esp_plan_query_cell(H, N: int, tolerance: float, opts: esp_plan_opts | None = None, **kw) -> dict:
    """Planner only for a triclinic cell (no GPU needed)."""
    if opts is None:
        opts = make_opts(**kw)
    cell = _cell(H)
    p = esp_plan_params()
    _check(load_library().esp_plan_query_cell(ctypes.byref(cell), int(N), float(tolerance), ctypes.byref(opts),
                                              ctypes.byref(p)))
    return p.as_dict()


def esp_influence_query(L_or_H, N: int, tolerance: float, opts: esp_plan_opts | None = None, **kw) -> np.ndarray:
    """The influence function p_k of the plan (host planner, no GPU needed), as
    an array [kz][ky][kx] over the half spectrum (kx in [0, n_f/2])."""
    if opts is None:
        opts = make_opts(**kw)
    lib = load_library()
    if np.ndim(L_or_H) == 2:
        box, cell = None, ctypes.byref(_cell(L_or_H))
    else:
        L = float(L_or_H)
        box, cell = ctypes.byref(esp_box((ctypes.c_double * 3)(L, L, L))), None
    n = ctypes.c_int64(0)
    _check(lib.esp_influence_query(box, cell, int(N), float(tolerance), ctypes.byref(opts), None, ctypes.byref(n)))
    out = np.zeros(n.value)
    _check(lib.esp_influence_query(box, cell, int(N), float(tolerance), ctypes.byref(opts),
                                   out.ctypes.data_as(_D), ctypes.byref(n)))
    n_f = round((2 * n.value) ** (1.0 / 3.0))
    while n_f * n_f * (n_f // 2 + 1) > n.value:
        n_f -= 1
    while n_f * n_f * (n_f // 2 + 1) < n.value:
        n_f += 1
    return out.reshape(n_f, n_f, n_f // 2 + 1)


def esp_set_exclusions(plan: int, pairs):
    """Pairs (n, 2) of caller indices whose direct interaction is removed
    from every compute that follows (None or an empty array clears them)."""
    arr = np.zeros((0, 2), dtype=np.int32) if pairs is None else \
        np.ascontiguousarray(np.asarray(pairs).reshape(-1, 2), dtype=np.int32)
    _check(load_library().esp_set_exclusions(_P(plan), arr.ctypes.data if len(arr) else None, int(len(arr))))


COULOMB_KJ_MOL_NM = 138.935458          # 1/(4 pi eps0) in kJ mol^-1 nm e^-2
MD_PREFACTOR = 4.0 * math.pi * COULOMB_KJ_MOL_NM   # plan prefactor for kJ/mol with the 1/(4 pi r) kernel


class MD:
    """Velocity-Verlet MD of flexible SPC/E-shaped water driven by a plan
    (esp_md_*). The plan must be cubic, hold (O, H, H) molecules, have its
    charges set and use prefactor MD_PREFACTOR."""

    def __init__(self, plan: int, xyz, vel, **params):
        lib = load_library()
        self.prm = esp_md_params()
        lib.esp_md_params_init(ctypes.byref(self.prm))
        for k, v in params.items():
            setattr(self.prm, k, v)
        x = np.ascontiguousarray(xyz, dtype=np.float64)
        v = np.ascontiguousarray(vel, dtype=np.float64)
        self.n = x.shape[0]
        out = _P()
        _check(lib.esp_md_create(_P(plan), ctypes.byref(self.prm), x.ctypes.data, v.ctypes.data, ctypes.byref(out)))
        self.handle = out.value

    def run(self, n_steps: int) -> np.ndarray:
        """(n_steps + 1, 4) energies: Coulomb, bonded, Lennard-Jones, kinetic (kJ/mol)."""
        e = np.zeros((n_steps + 1, 4))
        _check(load_library().esp_md_run(_P(self.handle), int(n_steps), e.ctypes.data))
        return e

    def state(self):
        x = np.zeros((self.n, 3))
        v = np.zeros((self.n, 3))
        _check(load_library().esp_md_state(_P(self.handle), x.ctypes.data, v.ctypes.data))
        return x, v

    def close(self):
        if self.handle:
            load_library().esp_md_destroy(_P(self.handle))
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def esp_plan_info(plan: int) -> dict:
    p = esp_plan_params()
    _check(load_library().esp_plan_info(_P(plan), ctypes.byref(p)))
    return p.as_dict()


def esp_set_charges(plan: int, q, where: int | None = None):
    ptr, w = _ptr(q)
    f32 = str(getattr(q, "dtype", "")).endswith("float32")
    fn = load_library().esp_set_charges_f32 if f32 else load_library().esp_set_charges
    _check(fn(_P(plan), ptr, where if where is not None else w))


def esp_set_positions(plan: int, xyz, where: int | None = None):
    ptr, w = _ptr(xyz)
    f32 = str(getattr(xyz, "dtype", "")).endswith("float32")
    fn = load_library().esp_set_positions_f32 if f32 else load_library().esp_set_positions
    _check(fn(_P(plan), ptr, where if where is not None else w))


def esp_step(plan: int, xyz, energy=None, forces=None, potential=None, where: int | None = None):
    """esp_set_positions(xyz) and esp_compute in one call (FP64 buffers: NumPy
    arrays or torch tensors, all host or all device)."""
    xp, xw = _ptr(xyz, np.float64 if isinstance(xyz, np.ndarray) else None)
    ws = {w for _, w in (_ptr(energy), _ptr(forces), _ptr(potential)) if w is not None} | {xw}
    if where is None:
        if len(ws) != 1:
            raise ValueError("esp_step needs all buffers on the host or all on the device")
        where = ws.pop()
    _check(load_library().esp_step(_P(plan), xp, _ptr(energy)[0], _ptr(forces)[0], _ptr(potential)[0], where))
    if isinstance(energy, np.ndarray):
        return float(energy[0])
    return None


def esp_compute(plan: int, energy=None, forces=None, potential=None, where: int | None = None):
    """Fill the given output buffers (NumPy float64 arrays, or torch tensors).

    With NumPy outputs, ``energy`` may be a length-1 float64 array. Returns the
    energy as a float when it was computed on the host.
    """
    ws = {w for _, w in (_ptr(energy), _ptr(forces), _ptr(potential)) if w is not None}
    if where is None:
        where = ws.pop() if len(ws) == 1 else ESP_HOST
    f32 = any(str(getattr(a, "dtype", "")).endswith("float32") for a in (forces, potential) if a is not None)
    e_ptr = _ptr(energy)[0]
    fn = load_library().esp_compute_f32 if f32 else load_library().esp_compute
    _check(fn(_P(plan), e_ptr, _ptr(forces)[0], _ptr(potential)[0], where))
    if isinstance(energy, np.ndarray):
        return float(energy[0])
    return None


def esp_synchronize(plan: int):
    _check(load_library().esp_synchronize(_P(plan)))


def esp_set_timing(plan: int, enable: int = 1):
    """0 off, 1 events around the phases, 2 events with the phases serialised."""
    _check(load_library().esp_set_timing(_P(plan), int(enable)))


PHASES = ("ingest_sort", "spread", "fft_r2c", "scale", "fft_c2r", "gather", "near", "finalize", "total")


def esp_phase_times(plan: int) -> dict:
    buf = (ctypes.c_float * len(PHASES))()
    _check(load_library().esp_phase_times(_P(plan), buf, len(PHASES)))
    return dict(zip(PHASES, list(buf)))


def esp_last_virial(plan: int) -> np.ndarray:
    """Virial of the last compute as a symmetric 3 x 3 array."""
    buf = (ctypes.c_double * 6)()
    _check(load_library().esp_last_virial(_P(plan), buf))
    xx, yy, zz, xy, xz, yz = list(buf)
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def esp_batch_last_virial(batch: int, n_systems: int) -> np.ndarray:
    """Virials of the last batch compute, shape (n_systems, 3, 3)."""
    buf = (ctypes.c_double * (6 * n_systems))()
    _check(load_library().esp_batch_last_virial(_P(batch), buf))
    v = np.array(list(buf)).reshape(n_systems, 6)
    out = np.empty((n_systems, 3, 3))
    for i, (xx, yy, zz, xy, xz, yz) in enumerate(v):
        out[i] = [[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]]
    return out


def esp_last_spectral_energy(plan: int) -> tuple[float, float]:
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load_library().esp_last_spectral_energy(_P(plan), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def esp_destroy(plan: int):
    _check(load_library().esp_destroy(_P(plan)))


def esp_local_part_static(L: float, N: int, tolerance: float, xyz, q, energy=None, forces=None,
                          potential=None, opts: esp_plan_opts | None = None, **kw):
    """Local part, self term and background without device allocation.

    xyz, q and the outputs are FP64 device buffers (torch CUDA tensors of
    3N, N, 1, 3N and N values, or raw device addresses); the work runs on
    opts.stream and the call returns once it has finished.
    """
    if opts is None:
        opts = make_opts(**kw)
    box = esp_box((ctypes.c_double * 3)(L, L, L))
    N = int(N)

    def dev_ptr(name, x, count, required):
        # raw device addresses (int) pass through to the library's own check
        if x is None:
            if required and N > 0:
                raise ValueError(f"{name} is required")
            return None
        if isinstance(x, int):
            return ctypes.c_void_p(x)
        if not (hasattr(x, "data_ptr") and getattr(x, "is_cuda", False)):
            raise TypeError(f"{name} must be a CUDA tensor (device memory), got {type(x).__name__}")
        if str(x.dtype) != "torch.float64":
            raise TypeError(f"{name} must be float64, got {x.dtype}")
        if x.numel() != count:
            raise ValueError(f"{name} must hold {count} values, got {x.numel()}")
        return _ptr(x)[0]

    _check(load_library().esp_local_part_static(
        ctypes.byref(box), N, float(tolerance), ctypes.byref(opts), dev_ptr("xyz", xyz, 3 * N, True),
        dev_ptr("q", q, N, True), dev_ptr("energy", energy, 1, False), dev_ptr("forces", forces, 3 * N, False),
        dev_ptr("potential", potential, N, False)))


def esp_autotune(L: float, tolerance: float, xyz, q, reps: int = 5, opts: esp_plan_opts | None = None,
                 **kw) -> tuple[dict, float]:
    """Time candidate shapes on this system; returns (chosen options, ms)."""
    if opts is None:
        opts = make_opts(**kw)
    pxyz, w = _ptr(xyz)
    pq, _ = _ptr(q)
    n = int(getattr(q, "shape", [len(q)])[0])
    box = esp_box((ctypes.c_double * 3)(L, L, L))
    out = esp_plan_opts()
    ms = ctypes.c_double()
    _check(load_library().esp_autotune(ctypes.byref(box), n, float(tolerance), ctypes.byref(opts), pxyz, pq,
                                       w, int(reps), ctypes.byref(out), ctypes.byref(ms)))
    chosen = {name: getattr(out, name) for name, _ in out._fields_ if name not in ("reserved", "stream")}
    return chosen, ms.value


def esp_batch_create(boxes, N, tolerance: float, opts: esp_plan_opts | None = None, **kw) -> int:
    """Batch of independent cubic systems: boxes[s] is the edge L of system s."""
    if opts is None:
        opts = make_opts(**kw)
    n = len(boxes)
    if len(N) != n:
        raise ValueError("boxes and N differ in length")
    arr = (esp_box * n)(*[esp_box((ctypes.c_double * 3)(L, L, L)) for L in boxes])
    counts = (ctypes.c_int64 * n)(*[int(x) for x in N])
    out = _P()
    _check(load_library().esp_batch_create(arr, counts, n, float(tolerance), ctypes.byref(opts),
                                           ctypes.byref(out)))
    return out.value


def esp_batch_query(boxes, N, tolerance: float, opts: esp_plan_opts | None = None, **kw) -> list:
    """Planner only (no GPU needed): per-system parameters esp_batch_create would choose."""
    if opts is None:
        opts = make_opts(**kw)
    n = len(boxes)
    arr = (esp_box * n)(*[esp_box((ctypes.c_double * 3)(L, L, L)) for L in boxes])
    counts = (ctypes.c_int64 * n)(*[int(x) for x in N])
    out = (esp_plan_params * n)()
    _check(load_library().esp_batch_query(arr, counts, n, float(tolerance), ctypes.byref(opts), out))
    return [out[i].as_dict() for i in range(n)]


def esp_batch_info(batch: int, sys: int) -> dict:
    p = esp_plan_params()
    _check(load_library().esp_batch_info(_P(batch), int(sys), ctypes.byref(p)))
    return p.as_dict()


def esp_batch_set_charges(batch: int, q, where: int | None = None):
    ptr, w = _ptr(q, np.float64 if isinstance(q, np.ndarray) else None)
    _check(load_library().esp_batch_set_charges(_P(batch), ptr, where if where is not None else w))


def esp_batch_compute(batch: int, xyz, energies=None, forces=None, potential=None, where: int | None = None):
    """FP64 buffers in the concatenated atom order; energies has one entry per system."""
    ptr, w = _ptr(xyz, np.float64 if isinstance(xyz, np.ndarray) else None)
    _check(load_library().esp_batch_compute(_P(batch), ptr, _ptr(energies)[0], _ptr(forces)[0],
                                            _ptr(potential)[0], where if where is not None else w))


def esp_batch_synchronize(batch: int):
    _check(load_library().esp_batch_synchronize(_P(batch)))


def esp_batch_set_timing(batch: int, enable: int = 1):
    _check(load_library().esp_batch_set_timing(_P(batch), int(enable)))


def esp_batch_phase_times(batch: int) -> dict:
    buf = (ctypes.c_float * len(PHASES))()
    _check(load_library().esp_batch_phase_times(_P(batch), buf, len(PHASES)))
    return dict(zip(PHASES, list(buf)))


def esp_batch_destroy(batch: int):
    _check(load_library().esp_batch_destroy(_P(batch)))


def esp_last_error() -> str:
    msg = load_library().esp_last_error()
    return msg.decode() if msg else ""


def esp_version() -> str:
    return load_library().esp_version().decode()


class Plan:
    """Owning handle: plan + host-side convenience (host arrays in, host arrays out)."""

    def __init__(self, L, N: int, tolerance: float, **opts):
        """L: cube edge, or a 3x3 box matrix (columns a, b, c) for a triclinic cell."""
        if np.ndim(L) == 2:
            self.handle = esp_plan_cell(L, N, tolerance, **opts)
        else:
            self.handle = esp_plan(L, N, tolerance, **opts)
        self.N = int(N)

    @property
    def info(self) -> dict:
        return esp_plan_info(self.handle)

    def set_charges(self, q, where=None):
        esp_set_charges(self.handle, q, where)

    def set_positions(self, xyz, where=None):
        esp_set_positions(self.handle, xyz, where)

    def set_exclusions(self, pairs):
        """Pairs (n, 2) of atom indices without direct interaction (None clears)."""
        esp_set_exclusions(self.handle, pairs)

    def compute(self):
        """Host arrays: returns (energy, forces (N,3), potential (N,))."""
        e = np.zeros(1)
        f = np.zeros((self.N, 3))
        u = np.zeros(self.N)
        esp_compute(self.handle, e, f, u, ESP_HOST)
        return float(e[0]), f, u

    def close(self):
        if self.handle:
            esp_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owning handle of a batch: host arrays in, host arrays out."""

    def __init__(self, boxes, N, tolerance: float, **opts):
        self.handle = esp_batch_create(boxes, N, tolerance, **opts)
        self.N = [int(x) for x in N]
        self.offsets = np.concatenate([[0], np.cumsum(self.N)]).astype(np.int64)

    def info(self, sys: int) -> dict:
        return esp_batch_info(self.handle, sys)

    def set_charges(self, q, where=None):
        esp_batch_set_charges(self.handle, q, where)

    def compute(self, xyz):
        """Returns (energies (S,), forces (sum N, 3), potential (sum N,))."""
        e = np.zeros(len(self.N))
        f = np.zeros((int(self.offsets[-1]), 3))
        u = np.zeros(int(self.offsets[-1]))
        esp_batch_compute(self.handle, np.ascontiguousarray(xyz, dtype=np.float64), e, f, u, ESP_HOST)
        return e, f, u

    def close(self):
        if self.handle:
            esp_batch_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def esp_server_opts_init() -> esp_server_opts:
    o = esp_server_opts()
    load_library().esp_server_opts_init(ctypes.byref(o))
    return o


def esp_server_create(r_c: float, **kw) -> int:
    o = esp_server_opts_init()
    o.r_c = float(r_c)
    for k, v in kw.items():
        setattr(o, k, v)
    out = _P()
    _check(load_library().esp_server_create(ctypes.byref(o), ctypes.byref(out)))
    return out.value


def esp_server_add_system(server: int, L: float, q) -> int:
    q = np.ascontiguousarray(q, dtype=np.float64)
    box = esp_box((ctypes.c_double * 3)(L, L, L))
    sid = ctypes.c_int()
    _check(load_library().esp_server_add_system(_P(server), ctypes.byref(box), int(q.shape[0]),
                                                _ptr(q)[0], ctypes.byref(sid)))
    return sid.value


def esp_server_submit(server: int, sid: int, tolerance: float, xyz) -> int:
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    t = ctypes.c_int64()
    _check(load_library().esp_server_submit(_P(server), int(sid), float(tolerance), _ptr(xyz)[0],
                                            ctypes.byref(t)))
    return t.value


def esp_server_poll(server: int, ticket: int) -> bool:
    d = ctypes.c_int()
    _check(load_library().esp_server_poll(_P(server), int(ticket), ctypes.byref(d)))
    return bool(d.value)


def esp_server_wait(server: int, ticket: int, n_atoms: int, timeout_ms: float = 0.0, forces: bool = True,
                    potential: bool = True):
    """Returns (energy, forces (N,3) or None, potential (N,) or None, latency ms)."""
    e = np.zeros(1)
    f = np.zeros((n_atoms, 3)) if forces else None
    u = np.zeros(n_atoms) if potential else None
    lat = ctypes.c_double()
    _check(load_library().esp_server_wait(_P(server), int(ticket), float(timeout_ms), _ptr(e)[0], _ptr(f)[0],
                                          _ptr(u)[0], ctypes.byref(lat)))
    return float(e[0]), f, u, lat.value


def esp_server_stats(server: int) -> dict:
    c = esp_server_counters()
    _check(load_library().esp_server_stats(_P(server), ctypes.byref(c)))
    return c.as_dict()


def esp_server_reset_stats(server: int):
    _check(load_library().esp_server_reset_stats(_P(server)))


def esp_server_destroy(server: int):
    _check(load_library().esp_server_destroy(_P(server)))


class Server:
    """Owning handle of a request server (host arrays in, host arrays out)."""

    def __init__(self, r_c: float, **opts):
        self.handle = esp_server_create(r_c, **opts)
        self.sizes = []

    def add_system(self, L: float, q) -> int:
        sid = esp_server_add_system(self.handle, L, q)
        self.sizes.append(int(np.asarray(q).shape[0]))
        return sid

    def submit(self, sid: int, tolerance: float, xyz) -> tuple:
        return esp_server_submit(self.handle, sid, tolerance, xyz), sid

    def wait(self, req: tuple, **kw):
        ticket, sid = req
        return esp_server_wait(self.handle, ticket, self.sizes[sid], **kw)

    def stats(self) -> dict:
        return esp_server_stats(self.handle)

    def close(self):
        if self.handle:
            esp_server_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
