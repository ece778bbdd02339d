"""ctypes binding of libndsi.so: the C-ABI entry points under the same names.

Argument marshalling only: every step of the path runs inside the library.  Array arguments may
be torch tensors (CUDA or CPU) or numpy arrays; they are passed as raw pointers.  The library
raises NdsiError when it is missing or a call fails; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libndsi.so")

NDSI_OK = 0
NDSI_ERR_INVALID = 1
NDSI_ERR_SINGULAR = 2
NDSI_ERR_OOM = 3
NDSI_ERR_CUDA = 4
NDSI_ERR_TIMEOUT = 5
NDSI_ERR_UNSUPPORTED = 6
NDSI_PREC_FP64 = 0
NDSI_PREC_SPLIT = 1
EXPORT = dict(perm_atoms=1, perm_basis=2, node_atoms=3, parent=4, struct_ptr=5, struct_atoms=6,
              level=7, schedule=8, tile_shapes=9)

# Every function declared in include/ndsi.h.
EXPORTED_SYMBOLS = (
    "ndsi_default_options", "ndsi_poles", "ndsi_analyze", "ndsi_plan_info", "ndsi_plan_export",
    "ndsi_factor_poles", "ndsi_selinv", "ndsi_density", "ndsi_plan_destroy",
    "ndsi_factors_destroy", "ndsi_last_error", "ndsi_profile_enable", "ndsi_profile_read",
    "ndsi_residue_sum_static", "ndsi_find_mu", "ndsi_mu_features", "ndsi_mlp_init",
    "ndsi_mlp_forward", "ndsi_mlp_grad", "ndsi_mlp_train", "ndsi_analyze_batched",
    "ndsi_density_batched", "ndsi_graph_enable", "ndsi_graph_info", "ndsi_autotune",
    "ndsi_density_energy", "ndsi_dos", "ndsi_factors_solve", "ndsi_eigenstates", "ndsi_mu_search",
    "ndsi_mu_search_batched", "ndsi_find_mu_batched", "ndsi_plan_check", "ndsi_density_poles",
    "ndsi_pole_shard", "ndsi_fp64_peak", "ndsi_density_batched_poles",
)
MU_EVAL_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_double))
MU_DOS_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                             ctypes.c_double, ctypes.POINTER(ctypes.c_double))
_PD = ctypes.POINTER(ctypes.c_double)
_PI = ctypes.POINTER(ctypes.c_int32)
MU_EVAL_BATCH_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, _PI, _PD, _PD)
MU_DOS_BATCH_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, _PI, _PD, ctypes.c_int32, _PD,
                                   _PD)
NDSI_MLP_INPUTS = 32
NDSI_MLP_HIDDEN = 64
NDSI_MLP_PARAMS = 6337


class NdsiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ndsi error {code}: {msg}")
        self.code = code


class ndsi_pattern(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p)]


class ndsi_options(ctypes.Structure):
    _fields_ = [("leaf_atoms", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("split_slices", ctypes.c_int32), ("block", ctypes.c_int32),
                ("m0_radius", ctypes.c_double), ("max_workspace_bytes", ctypes.c_int64),
                ("outer_block", ctypes.c_int32), ("split_bands", ctypes.c_int32),
                ("cell", ctypes.c_double * 3), ("screen_degree", ctypes.c_int32),
                ("split_far_ratio", ctypes.c_double)]


class ndsi_plan_summary(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("n_atoms", ctypes.c_int32),
                ("n_nodes", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("max_front", ctypes.c_int32), ("front_elems", ctypes.c_int64),
                ("flops_per_pole", ctypes.c_double), ("bytes_per_pole", ctypes.c_double),
                ("n_launches", ctypes.c_int32), ("n_systems", ctypes.c_int32),
                ("split_slices", ctypes.c_int32), ("split_bands", ctypes.c_int32)]


class ndsi_profile_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double),
                ("tensor_flops", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libndsi.so (build it first with paper_1005_0088_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise NdsiError(-1, f"{path} is missing: run paper_1005_0088_gb300.build.build() "
                            "(the CUDA library is required; there is no fallback)")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.ndsi_default_options.argtypes = [ctypes.POINTER(ndsi_options)]
    lib.ndsi_default_options.restype = None
    lib.ndsi_poles.argtypes = [i32, vp, vp]
    lib.ndsi_analyze.argtypes = [ctypes.POINTER(ndsi_pattern), i32, vp, vp,
                                 ctypes.POINTER(ndsi_options), ctypes.POINTER(vp)]
    lib.ndsi_plan_info.argtypes = [vp, ctypes.POINTER(ndsi_plan_summary)]
    lib.ndsi_plan_export.argtypes = [vp, i32, vp]
    lib.ndsi_factor_poles.argtypes = [vp, vp, vp, vp, i32, ctypes.POINTER(vp), vp]
    lib.ndsi_selinv.argtypes = [vp, vp, vp]
    lib.ndsi_density.argtypes = [vp, vp, vp, dbl, dbl, i32, vp, vp, vp]
    lib.ndsi_density_poles.argtypes = [vp, vp, vp, dbl, dbl, i32, i32, i32, i32, vp, vp, vp]
    lib.ndsi_density_poles.restype = ctypes.c_int
    lib.ndsi_pole_shard.argtypes = [i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.ndsi_pole_shard.restype = ctypes.c_int
    lib.ndsi_density_batched_poles.argtypes = [vp, vp, vp, vp, vp, i32, i32, i32, i32, vp, vp, vp]
    lib.ndsi_density_batched_poles.restype = ctypes.c_int
    lib.ndsi_fp64_peak.argtypes = [ctypes.POINTER(dbl), vp]
    lib.ndsi_fp64_peak.restype = ctypes.c_int
    lib.ndsi_plan_destroy.argtypes = [vp]
    lib.ndsi_plan_destroy.restype = None
    lib.ndsi_factors_destroy.argtypes = [vp]
    lib.ndsi_factors_destroy.restype = None
    lib.ndsi_profile_enable.argtypes = [vp, i32]
    lib.ndsi_graph_enable.argtypes = [vp, i32]
    lib.ndsi_density_energy.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, i32, vp, vp, vp, vp]
    lib.ndsi_density_energy.restype = ctypes.c_int
    lib.ndsi_dos.argtypes = [vp, vp, vp, vp, i32, ctypes.c_double, vp, vp]
    lib.ndsi_dos.restype = ctypes.c_int
    lib.ndsi_mu_search.argtypes = [MU_EVAL_FN, MU_DOS_FN, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, i32, ctypes.c_double, ctypes.c_double, ctypes.c_double, i32,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(i32)]
    lib.ndsi_mu_search.restype = ctypes.c_int
    lib.ndsi_mu_search_batched.argtypes = [i32, MU_EVAL_BATCH_FN, MU_DOS_BATCH_FN, vp, vp, vp, vp, vp, i32, vp, vp,
                                           ctypes.c_double, i32, vp, vp, vp, ctypes.POINTER(i32)]
    lib.ndsi_mu_search_batched.restype = ctypes.c_int
    lib.ndsi_find_mu_batched.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, ctypes.c_double, i32, vp, vp, vp,
                                         ctypes.POINTER(i32), vp]
    lib.ndsi_find_mu_batched.restype = ctypes.c_int
    lib.ndsi_plan_check.argtypes = [vp]
    lib.ndsi_plan_check.restype = ctypes.c_int
    lib.ndsi_factors_solve.argtypes = [vp, i32, vp, i32, vp, vp]
    lib.ndsi_factors_solve.restype = ctypes.c_int
    lib.ndsi_eigenstates.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, i32, i32, i32,
                                     ctypes.c_double, ctypes.c_uint64, vp, vp, vp, ctypes.POINTER(i32), vp]
    lib.ndsi_eigenstates.restype = ctypes.c_int
    lib.ndsi_autotune.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, i32,
                                  ctypes.POINTER(i32), ctypes.POINTER(i32), vp]
    lib.ndsi_autotune.restype = ctypes.c_int
    lib.ndsi_graph_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.ndsi_graph_enable.restype = ctypes.c_int
    lib.ndsi_graph_info.restype = ctypes.c_int
    lib.ndsi_profile_read.argtypes = [vp, ctypes.POINTER(ndsi_profile_entry), i32,
                                      ctypes.POINTER(i32)]
    lib.ndsi_residue_sum_static.argtypes = [vp, vp, i32, vp, i64, vp, vp, vp]
    lib.ndsi_residue_sum_static.restype = ctypes.c_int
    lib.ndsi_find_mu.argtypes = [vp, vp, vp, dbl, i32, dbl, dbl, dbl, dbl, i32, vp,
                                 ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(i32), vp]
    lib.ndsi_find_mu.restype = ctypes.c_int
    lib.ndsi_mu_features.argtypes = [vp, vp, vp, dbl, dbl, i32, ctypes.c_uint64, vp, vp]
    lib.ndsi_mlp_init.argtypes = [vp, ctypes.c_uint64, vp]
    lib.ndsi_mlp_forward.argtypes = [vp, vp, i32, vp, vp]
    lib.ndsi_mlp_grad.argtypes = [vp, vp, vp, i32, vp, vp, vp]
    lib.ndsi_mlp_train.argtypes = [vp, vp, vp, i32, i32, ctypes.c_float, vp, vp]
    for name in ("ndsi_mu_features", "ndsi_mlp_init", "ndsi_mlp_forward", "ndsi_mlp_grad",
                 "ndsi_mlp_train"):
        getattr(lib, name).restype = ctypes.c_int
    lib.ndsi_analyze_batched.argtypes = [i32, vp, vp, vp, vp, ctypes.POINTER(ndsi_options),
                                         ctypes.POINTER(vp)]
    lib.ndsi_density_batched.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, vp]
    lib.ndsi_analyze_batched.restype = ctypes.c_int
    lib.ndsi_density_batched.restype = ctypes.c_int
    lib.ndsi_last_error.argtypes = []
    lib.ndsi_last_error.restype = ctypes.c_char_p
    for name in ("ndsi_poles", "ndsi_analyze", "ndsi_plan_info", "ndsi_plan_export",
                 "ndsi_factor_poles", "ndsi_selinv", "ndsi_density", "ndsi_profile_enable",
                 "ndsi_profile_read"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc):
    if rc != NDSI_OK:
        raise NdsiError(rc, load().ndsi_last_error().decode())


def _ptr(x):
    """Raw address of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("contiguous tensor required")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("contiguous array required")
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(type(x))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def ndsi_default_options():
    """The library's default ndsi_options."""
    o = ndsi_options()
    load().ndsi_default_options(ctypes.byref(o))
    return o


def ndsi_poles(M: int):
    """(z, R): poles and residues of the Eq. 7 fraction with M pole pairs (host)."""
    z = np.zeros(M)
    R = np.zeros(M)
    _check(load().ndsi_poles(int(M), _ptr(z), _ptr(R)))
    return z, R


class Plan:
    """Owner of an ndsi_plan handle."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ndsi_plan_destroy(self.handle)
            self.handle = None


class Factors:
    """Owner of an ndsi_factors handle (keeps its plan alive)."""

    def __init__(self, handle, plan, n_poles):
        self.handle = handle
        self.plan = plan
        self.n_poles = n_poles

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ndsi_factors_destroy(self.handle)
            self.handle = None


def ndsi_analyze(n, rowptr, col, n_atoms, centers, atom_of_basis, options=None) -> Plan:
    """ndsi_analyze: nested dissection, supernodes and schedule of one pattern (host only)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    centers = np.ascontiguousarray(centers, dtype=np.float64)
    aob = np.ascontiguousarray(atom_of_basis, dtype=np.int32)
    pat = ndsi_pattern(int(n), rowptr.ctypes.data, col.ctypes.data)
    opt = options if options is not None else ndsi_default_options()
    h = ctypes.c_void_p()
    _check(load().ndsi_analyze(ctypes.byref(pat), int(n_atoms), _ptr(centers), _ptr(aob),
                               ctypes.byref(opt), ctypes.byref(h)))
    return Plan(h)


def ndsi_plan_info(plan: Plan) -> dict:
    """ndsi_plan_info as a dict of the ndsi_plan_summary fields."""
    s = ndsi_plan_summary()
    _check(load().ndsi_plan_info(plan.handle, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in ndsi_plan_summary._fields_}


def ndsi_plan_check(plan: Plan) -> None:
    """Raise NdsiError if the plan's schedule would index out of bounds or race (host only)."""
    _check(load().ndsi_plan_check(plan.handle))


def ndsi_plan_export(plan: Plan, what: str) -> np.ndarray:
    """One structure table of the plan (perm_atoms, perm_basis, node_atoms, parent, struct_ptr,
    struct_atoms, schedule, tile_shapes) as a numpy array."""
    info = ndsi_plan_info(plan)
    nn = info["n_nodes"]
    if what == "struct_atoms":
        ptr = ndsi_plan_export(plan, "struct_ptr")
        out = np.zeros(max(int(ptr[-1]), 1), dtype=np.int32)
        _check(load().ndsi_plan_export(plan.handle, EXPORT[what], _ptr(out)))
        return out[:int(ptr[-1])]
    sizes = dict(perm_atoms=(info["n_atoms"], np.int32), perm_basis=(info["n"], np.int32),
                 node_atoms=(nn + 1, np.int32), parent=(nn, np.int32),
                 struct_ptr=(nn + 1, np.int64), level=(nn, np.int32),
                 schedule=(4 * info["n_launches"], np.int32), tile_shapes=(info["n_launches"], np.int32))
    cnt, dt = sizes[what]
    out = np.zeros(cnt, dtype=dt)
    _check(load().ndsi_plan_export(plan.handle, EXPORT[what], _ptr(out)))
    if what == "schedule":
        return out.reshape(-1, 4)
    return out


def ndsi_factor_poles(plan: Plan, H, S, z, stream=None) -> Factors:
    """Factor z_p S - H for every point of z (complex array); returns the factors handle."""
    z = np.ascontiguousarray(np.asarray(z, dtype=np.complex128))
    zz = np.ascontiguousarray(z.view(np.float64))
    h = ctypes.c_void_p()
    _check(load().ndsi_factor_poles(plan.handle, _ptr(H), _ptr(S), _ptr(zz), int(z.shape[0]),
                                    ctypes.byref(h), _stream(stream)))
    return Factors(h, plan, int(z.shape[0]))


def ndsi_selinv(factors: Factors, G_out=None, stream=None):
    """Selected inversion of the factors; G_out (n_poles x nnz x 2 doubles) or None."""
    _check(load().ndsi_selinv(factors.handle, _ptr(G_out), _stream(stream)))
    return G_out


def ndsi_density(plan: Plan, H, S, mu, kT, n_poles, rho_out, n_elec_out=None, stream=None):
    """rho on the pattern and Tr(rho S) at (mu, kT) with n_poles poles (Eq. 8, Eq. 40)."""
    _check(load().ndsi_density(plan.handle, _ptr(H), _ptr(S), float(mu), float(kT), int(n_poles),
                               _ptr(rho_out), _ptr(n_elec_out), _stream(stream)))
    return rho_out


def ndsi_density_poles(plan: Plan, H, S, mu, kT, n_poles, pole_begin, pole_end, with_m0, rho_out,
                       n_elec_out=None, stream=None):
    """One rank's share of Eq. 8: M0 (if with_m0) plus the poles pole_begin <= p < pole_end of an
    n_poles expansion, and its Tr(rho_part S)."""
    _check(load().ndsi_density_poles(plan.handle, _ptr(H), _ptr(S), float(mu), float(kT), int(n_poles),
                                     int(pole_begin), int(pole_end), int(bool(with_m0)), _ptr(rho_out),
                                     _ptr(n_elec_out), _stream(stream)))
    return rho_out


def ndsi_pole_shard(n_poles, rank, world):
    """(pole_begin, pole_end, with_m0) of `rank` among `world` processes (host only)."""
    b, e, m = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().ndsi_pole_shard(int(n_poles), int(rank), int(world), ctypes.byref(b), ctypes.byref(e),
                                  ctypes.byref(m)))
    return b.value, e.value, bool(m.value)


def ndsi_fp64_peak(stream=None):
    """Measured FP64 (DFMA) throughput of the current GPU in TFLOP/s."""
    out = ctypes.c_double()
    _check(load().ndsi_fp64_peak(ctypes.byref(out), _stream(stream)))
    return out.value


def ndsi_density_energy(plan: Plan, H, S, mu, kT, n_poles, rho_out, e_out, n_elec_out=None, stream=None):
    """rho and the energy density matrix (Eq. 10) on the pattern in one sweep."""
    _check(load().ndsi_density_energy(plan.handle, _ptr(H), _ptr(S), float(mu), float(kT), int(n_poles),
                                      _ptr(rho_out), _ptr(e_out), _ptr(n_elec_out), _stream(stream)))
    return rho_out, e_out


def ndsi_dos(plan: Plan, H, S, energies, eta, stream=None):
    """D(E) = -(2/pi) Im Tr(G(E + i eta) S) at each energy (Eq. 41); returns a host array."""
    E = np.ascontiguousarray(np.asarray(energies, dtype=np.float64).reshape(-1))
    D = np.zeros_like(E)
    _check(load().ndsi_dos(plan.handle, _ptr(H), _ptr(S), _ptr(E), int(E.size), float(eta), _ptr(D),
                           _stream(stream)))
    return D


def ndsi_mu_search(delta_n, elo, ehi, kT, n_electrons, dos=None, n_grid=0, mu_lo=0.0, mu_hi=0.0,
                   tol_electrons=1e-8, max_iter=100):
    """(mu, DeltaN, evaluations) of the host chemical-potential search over Python callables:
    delta_n(mu) -> float and, optionally, dos(E: ndarray, eta) -> ndarray.  Raises NdsiError
    (with .result = (mu, DeltaN, evaluations)) when the search fails."""
    failure = []

    def ev(_ctx, mu, out):
        try:
            out[0] = float(delta_n(mu))
            return 0
        except Exception as exc:  # noqa: BLE001 - reported after the search returns
            failure.append(exc)
            return NDSI_ERR_INVALID

    def ds(_ctx, E, n, eta, out):
        try:
            D = np.asarray(dos(np.ctypeslib.as_array(E, shape=(n,)).copy(), eta), dtype=np.float64)
            for k in range(n):
                out[k] = float(D[k])
            return 0
        except Exception as exc:  # noqa: BLE001
            failure.append(exc)
            return NDSI_ERR_INVALID

    ev_c = MU_EVAL_FN(ev)
    ds_c = MU_DOS_FN(ds) if dos is not None else ctypes.cast(None, MU_DOS_FN)
    mu, dn, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    rc = load().ndsi_mu_search(ev_c, ds_c, None, float(elo), float(ehi), float(kT), float(n_electrons),
                               int(n_grid), float(mu_lo), float(mu_hi), float(tol_electrons), int(max_iter),
                               ctypes.byref(mu), ctypes.byref(dn), ctypes.byref(it))
    if failure:
        raise failure[0]
    if rc != NDSI_OK:
        err = NdsiError(rc, load().ndsi_last_error().decode())
        err.result = (mu.value, dn.value, it.value)
        raise err
    return mu.value, dn.value, it.value


def ndsi_mu_search_batched(delta_n, elo, ehi, kT, n_electrons, dos=None, n_grid=0, mu_lo=None, mu_hi=None,
                           tol_electrons=1e-8, max_iter=100):
    """Lockstep searches for several systems over Python callables answering whole rounds:
    delta_n(mu: ndarray, active: ndarray) -> ndarray and, optionally,
    dos(E: ndarray (systems x n), eta: ndarray, active) -> ndarray.  Returns
    (mu, DeltaN, evaluations per system, rounds)."""
    elo, ehi, kT, ne = (np.ascontiguousarray(np.asarray(v, dtype=np.float64)) for v in (elo, ehi, kT, n_electrons))
    ns = elo.size
    lo = None if mu_lo is None else np.ascontiguousarray(np.asarray(mu_lo, dtype=np.float64))
    hi = None if mu_hi is None else np.ascontiguousarray(np.asarray(mu_hi, dtype=np.float64))
    failure = []

    def ev(_ctx, n, active, mu, out):
        try:
            d = np.asarray(delta_n(np.ctypeslib.as_array(mu, shape=(n,)).copy(),
                                   np.ctypeslib.as_array(active, shape=(n,)).copy()), dtype=np.float64)
            for s_ in range(n):
                out[s_] = float(d[s_])
            return 0
        except Exception as exc:  # noqa: BLE001
            failure.append(exc)
            return NDSI_ERR_INVALID

    def ds(_ctx, n, active, E, m, eta, out):
        try:
            D = np.asarray(dos(np.ctypeslib.as_array(E, shape=(n, m)).copy(),
                               np.ctypeslib.as_array(eta, shape=(n,)).copy(),
                               np.ctypeslib.as_array(active, shape=(n,)).copy()), dtype=np.float64).reshape(-1)
            for k in range(n * m):
                out[k] = float(D[k])
            return 0
        except Exception as exc:  # noqa: BLE001
            failure.append(exc)
            return NDSI_ERR_INVALID

    ev_c = MU_EVAL_BATCH_FN(ev)
    ds_c = MU_DOS_BATCH_FN(ds) if dos is not None else ctypes.cast(None, MU_DOS_BATCH_FN)
    mu, dn = np.zeros(ns), np.zeros(ns)
    evals = np.zeros(ns, dtype=np.int32)
    rounds = ctypes.c_int32()
    rc = load().ndsi_mu_search_batched(ns, ev_c, ds_c, None, _ptr(elo), _ptr(ehi), _ptr(kT), _ptr(ne), int(n_grid),
                                       _ptr(lo), _ptr(hi), float(tol_electrons), int(max_iter), _ptr(mu), _ptr(dn),
                                       _ptr(evals), ctypes.byref(rounds))
    if failure:
        raise failure[0]
    if rc != NDSI_OK:
        err = NdsiError(rc, load().ndsi_last_error().decode())
        err.result = (mu, dn, evals, rounds.value)
        raise err
    return mu, dn, evals, rounds.value


def ndsi_factors_solve(factors, pole, Y, X_out, stream=None):
    """X = (z_p S - H)^{-1} Y with the factors of pole p; Y, X complex (n, k) or (n,), C order."""
    k = 1 if Y.ndim == 1 else int(Y.shape[1])
    _check(load().ndsi_factors_solve(factors.handle, int(pole), _ptr(Y), k, _ptr(X_out), _stream(stream)))
    return X_out


def ndsi_eigenstates(plan: Plan, H, S, xi, n_states, eta=1e-3, block=None, max_iter=200, tol=1e-10,
                     seed=12345, C_out=None, stream=None):
    """(eps, C, residuals, iterations): the n_states eigenpairs nearest xi (App. B).

    C is (n_states, n), a host array unless a device tensor C_out is given."""
    block = int(block if block is not None else min(32, n_states + 4))
    eps = np.zeros(n_states)
    res = np.zeros(n_states)
    it = ctypes.c_int32()
    if C_out is None:
        C_out = np.zeros((n_states, int(ndsi_plan_info(plan)["n"])))
    _check(load().ndsi_eigenstates(plan.handle, _ptr(H), _ptr(S), float(xi), float(eta), int(n_states), block,
                                   int(max_iter), float(tol), int(seed), _ptr(eps), _ptr(C_out), _ptr(res),
                                   ctypes.byref(it), _stream(stream)))
    return eps, C_out, res, it.value


def _options(options):
    """ndsi_options from keyword values (cell as a 3-sequence)."""
    opt = ndsi_default_options()
    for k, v in options.items():
        if k == "cell":
            v = (ctypes.c_double * 3)(*[float(c) for c in v])
        setattr(opt, k, v)
    return opt


def analyze_system(system, **options) -> Plan:
    """ndsi_analyze on a synth.System-like object (fields n, rowptr, col, centers, atom_of_basis)."""
    opt = _options(options)
    return ndsi_analyze(system.n, system.rowptr, system.col, system.centers.shape[0],
                        system.centers, system.atom_of_basis, opt)


def ndsi_autotune(plan: Plan, H, S, mu, kT, n_poles, stream=None):
    """Per-step choice between tensor-core and FP64 GEMMs by timing; returns (n_split, n_fp64)."""
    ns = ctypes.c_int32(0)
    nf = ctypes.c_int32(0)
    _check(load().ndsi_autotune(plan.handle, _ptr(H), _ptr(S), float(mu), float(kT), int(n_poles),
                                ctypes.byref(ns), ctypes.byref(nf), _stream(stream)))
    return ns.value, nf.value


def ndsi_graph_enable(plan: Plan, enable: bool = True):
    """Run density sweeps as one captured CUDA graph (default) or as direct launches."""
    _check(load().ndsi_graph_enable(plan.handle, 1 if enable else 0))


def ndsi_graph_info(plan: Plan) -> int:
    """Kernel nodes of the plan's captured sweep (0 when none is held)."""
    n = ctypes.c_int64(0)
    _check(load().ndsi_graph_info(plan.handle, ctypes.byref(n)))
    return n.value


def ndsi_profile_enable(plan: Plan, enable=True, by_level: bool = False):
    """Per-kernel timing on (by_level splits GEMM and slicing families by tree level) or off."""
    _check(load().ndsi_profile_enable(plan.handle, (2 if by_level else 1) if enable else 0))


def ndsi_profile_read(plan: Plan) -> dict:
    """{family: dict(launches, ms, flops, bytes)} accumulated since ndsi_profile_enable."""
    cap = 1024
    buf = (ndsi_profile_entry * cap)()
    n = ctypes.c_int32()
    _check(load().ndsi_profile_read(plan.handle, buf, cap, ctypes.byref(n)))
    return {buf[i].name.decode(): dict(launches=buf[i].launches, ms=buf[i].ms, flops=buf[i].flops,
                                       bytes=buf[i].bytes, tensor_flops=buf[i].tensor_flops)
            for i in range(n.value)}


def ndsi_residue_sum_static(G, c, n_points, S, nnz, rho_out, n_elec_out=None, stream=None):
    """rho and Tr(rho S) from caller-held G without any device allocation (device arrays only)."""
    _check(load().ndsi_residue_sum_static(_ptr(G), _ptr(c), int(n_points), _ptr(S), int(nnz),
                                          _ptr(rho_out), _ptr(n_elec_out), _stream(stream)))
    return rho_out


def ndsi_find_mu(plan: Plan, H, S, kT, n_poles, n_electrons, rho_out, mu_lo=0.0, mu_hi=0.0,
                 tol_electrons=1e-8, max_iter=100, stream=None):
    """(mu, N_e, evaluations): Eq. 40 solved by bracketed interpolation/bisection."""
    mu = ctypes.c_double()
    ne = ctypes.c_double()
    it = ctypes.c_int32()
    _check(load().ndsi_find_mu(plan.handle, _ptr(H), _ptr(S), float(kT), int(n_poles),
                               float(n_electrons), float(mu_lo), float(mu_hi), float(tol_electrons),
                               int(max_iter), _ptr(rho_out), ctypes.byref(mu), ctypes.byref(ne),
                               ctypes.byref(it), _stream(stream)))
    return mu.value, ne.value, it.value


def ndsi_find_mu_batched(plan: Plan, H, S, kT, n_poles, n_electrons, rho_out, mu_lo=None, mu_hi=None,
                         tol_electrons=1e-8, max_iter=100, stream=None):
    """(mu[], N_e[], rounds): Eq. 40 for every system of a batched plan, searched in lockstep."""
    kT = np.ascontiguousarray(np.asarray(kT, dtype=np.float64))
    ne = np.ascontiguousarray(np.asarray(n_electrons, dtype=np.float64))
    lo = None if mu_lo is None else np.ascontiguousarray(np.asarray(mu_lo, dtype=np.float64))
    hi = None if mu_hi is None else np.ascontiguousarray(np.asarray(mu_hi, dtype=np.float64))
    mu, ne_out = np.zeros(kT.size), np.zeros(kT.size)
    rounds = ctypes.c_int32()
    _check(load().ndsi_find_mu_batched(plan.handle, _ptr(H), _ptr(S), _ptr(kT), int(n_poles), _ptr(ne), _ptr(lo),
                                       _ptr(hi), float(tol_electrons), int(max_iter), _ptr(rho_out), _ptr(mu),
                                       _ptr(ne_out), ctypes.byref(rounds), _stream(stream)))
    return mu, ne_out, rounds.value


def ndsi_mu_features(plan: Plan, H, S, n_electrons, kT, feat_out, n_vectors=16, seed=12345,
                     stream=None):
    """The 32 spectral-moment features of (H, S) for the chemical-potential seed network."""
    _check(load().ndsi_mu_features(plan.handle, _ptr(H), _ptr(S), float(n_electrons), float(kT),
                                   int(n_vectors), int(seed), _ptr(feat_out), _stream(stream)))
    return feat_out


def ndsi_mlp_init(params, seed=0, stream=None):
    """Glorot-uniform initial parameters of the seed network (device float array)."""
    _check(load().ndsi_mlp_init(_ptr(params), int(seed), _stream(stream)))
    return params


def ndsi_mlp_forward(params, X, n, Y, stream=None):
    """Network outputs Y[s] for the rows of X (device arrays)."""
    _check(load().ndsi_mlp_forward(_ptr(params), _ptr(X), int(n), _ptr(Y), _stream(stream)))
    return Y


def ndsi_mlp_grad(params, X, T, n, grad, loss=None, stream=None):
    """Gradient of the mean squared error over the n rows (and the loss, if given)."""
    _check(load().ndsi_mlp_grad(_ptr(params), _ptr(X), _ptr(T), int(n), _ptr(grad), _ptr(loss),
                                _stream(stream)))
    return grad


def ndsi_mlp_train(params, X, T, n, steps, lr, stream=None):
    """Full-batch Adam on the mean squared error; returns the final loss."""
    loss = np.zeros(1, dtype=np.float32)
    _check(load().ndsi_mlp_train(_ptr(params), _ptr(X), _ptr(T), int(n), int(steps), float(lr),
                                 _ptr(loss), _stream(stream)))
    return float(loss[0])


def analyze_batched(systems, **options) -> Plan:
    """ndsi_analyze_batched over synth.System-like objects."""
    opt = _options(options)
    ns = len(systems)
    keep = []
    pats = (ndsi_pattern * ns)()
    na = np.zeros(ns, dtype=np.int32)
    cen_ptrs = (ctypes.c_void_p * ns)()
    aob_ptrs = (ctypes.c_void_p * ns)()
    for i, sy in enumerate(systems):
        rp = np.ascontiguousarray(sy.rowptr, dtype=np.int64)
        cl = np.ascontiguousarray(sy.col, dtype=np.int32)
        ce = np.ascontiguousarray(sy.centers, dtype=np.float64)
        ab = np.ascontiguousarray(sy.atom_of_basis, dtype=np.int32)
        keep += [rp, cl, ce, ab]
        pats[i] = ndsi_pattern(int(sy.n), rp.ctypes.data, cl.ctypes.data)
        na[i] = sy.centers.shape[0]
        cen_ptrs[i] = ce.ctypes.data
        aob_ptrs[i] = ab.ctypes.data
    h = ctypes.c_void_p()
    _check(load().ndsi_analyze_batched(ns, pats, _ptr(na), cen_ptrs, aob_ptrs, ctypes.byref(opt),
                                       ctypes.byref(h)))
    return Plan(h)


def ndsi_density_batched(plan: Plan, H, S, mu, kT, n_poles, rho_out, n_elec_out=None, stream=None):
    """rho and Tr(rho S) of every system of a batched plan at its own mu and kT."""
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    kT = np.ascontiguousarray(kT, dtype=np.float64)
    _check(load().ndsi_density_batched(plan.handle, _ptr(H), _ptr(S), _ptr(mu), _ptr(kT),
                                       int(n_poles), _ptr(rho_out), _ptr(n_elec_out),
                                       _stream(stream)))
    return rho_out


def ndsi_density_batched_poles(plan: Plan, H, S, mu, kT, n_poles, pole_begin, pole_end, with_m0, rho_out,
                               n_elec_out=None, stream=None):
    """One rank's share (poles pole_begin..pole_end-1, M0 if with_m0) of ndsi_density_batched."""
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    kT = np.ascontiguousarray(kT, dtype=np.float64)
    _check(load().ndsi_density_batched_poles(plan.handle, _ptr(H), _ptr(S), _ptr(mu), _ptr(kT),
                                             int(n_poles), int(pole_begin), int(pole_end),
                                             int(bool(with_m0)), _ptr(rho_out), _ptr(n_elec_out),
                                             _stream(stream)))
    return rho_out
