"""ctypes binding of libgbmc.so, the C ABI declared in include/gbmc.h.

Argument marshalling only: every function forwards to the C entry point of the
same name. Device buffers are torch CUDA tensors (their data_ptr is passed);
host buffers are numpy arrays. Streams are raw cudaStream_t handles (an int,
e.g. ``torch.cuda.current_stream().cuda_stream``) or None for the default
stream. A missing or unloadable library raises immediately: there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GBMC_LIBRARY=libgbmc_check.so selects the bounds-checked build (same directory)
LIB_PATH = os.path.join(_HERE, os.path.basename(os.environ.get("GBMC_LIBRARY", "libgbmc.so")))
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "gbmc.h")

GBMC_OK, GBMC_ERR_ARG, GBMC_ERR_OOM, GBMC_ERR_CUDA, GBMC_ERR_TIMEOUT, GBMC_ERR_STATE = 0, -1, -2, -3, -4, -5
GBMC_ISING_FM, GBMC_EA_PMJ = 0, 1
GBMC_INT8, GBMC_BITPACK = 0, 1
GBMC_START_ALL_UP, GBMC_START_RANDOM = 0, 1
GBMC_SCHED_LINEAR, GBMC_SCHED_LIST, GBMC_SCHED_BISECTION, GBMC_SCHED_MLP = 0, 1, 2, 3
GBMC_LAUNCH_AUTO, GBMC_LAUNCH_GRID, GBMC_LAUNCH_PERSISTENT = 0, 1, 2
GBMC_KERNEL_AUTO, GBMC_KERNEL_BYTES, GBMC_KERNEL_BITS = 0, 1, 2
GBMC_RESAMPLE_MULTINOMIAL, GBMC_RESAMPLE_NEAREST, GBMC_RESAMPLE_POISSON = 0, 1, 2
GBMC_RNG_PHILOX, GBMC_RNG_MSC = 0, 1


class GbmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("gbmc status %d: %s" % (status, msg))
        self.status = status


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_uint64), ("total_ms", C.c_double)]


class Tuning(C.Structure):
    _fields_ = [("resident", C.c_int32), ("threads_per_copy", C.c_uint32), ("copies_per_cta", C.c_uint32),
                ("row_walk", C.c_int32), ("ms_per_sweep", C.c_double), ("n_candidates", C.c_uint32),
                ("persistent", C.c_int32), ("kernel", C.c_int32)]


class ScheduleRecord(C.Structure):
    _fields_ = [("beta", C.c_double), ("dbeta", C.c_double), ("alpha", C.c_double), ("proposal", C.c_double),
                ("alpha_proposal", C.c_double), ("var", C.c_double), ("features", C.c_float * 6),
                ("kind", C.c_int32), ("clamped", C.c_int32), ("evals", C.c_int32), ("pad", C.c_int32)]


class LatticeDesc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("L", C.c_int32), ("model", C.c_int32), ("layout", C.c_int32),
                ("start", C.c_int32), ("n_instances", C.c_uint32), ("n_replicas", C.c_uint32),
                ("instance_base", C.c_uint32), ("seed", C.c_uint64)]


class LatticeInfo(C.Structure):
    _fields_ = [("n_sites", C.c_int64), ("n_copies", C.c_int64), ("spin_bytes", C.c_int64),
                ("sweep_counter", C.c_uint32), ("pad", C.c_uint32), ("spins_dev", C.c_void_p)]


class PaConfig(C.Structure):
    _fields_ = [("theta", C.c_uint32), ("n_steps", C.c_uint32), ("schedule", C.c_int32), ("init", C.c_int32),
                ("beta_f", C.c_double), ("betas", C.c_void_p), ("target_overlap", C.c_double),
                ("dbeta_max", C.c_double), ("mlp_params", C.c_void_p), ("overlap_lo", C.c_double),
                ("overlap_hi", C.c_double), ("resample", C.c_int32), ("initial_replicas", C.c_uint32),
                ("sweep_rng", C.c_int32), ("pad", C.c_int32)]


class PaStats(C.Structure):
    _fields_ = [("beta", C.c_double), ("dbeta", C.c_double), ("lnQ", C.c_double), ("lnZ", C.c_double),
                ("sumE", C.c_int64), ("sumE2", C.c_int64), ("sumAbsM", C.c_int64), ("sumM2", C.c_int64),
                ("Emin", C.c_int32), ("Emax", C.c_int32), ("step", C.c_uint32), ("n_replicas", C.c_uint32),
                ("overlap", C.c_double), ("proposal_kind", C.c_int32), ("pad", C.c_int32)]


PA_STATS_DTYPE = np.dtype([("beta", "<f8"), ("dbeta", "<f8"), ("lnQ", "<f8"), ("lnZ", "<f8"),
                           ("sumE", "<i8"), ("sumE2", "<i8"), ("sumAbsM", "<i8"), ("sumM2", "<i8"),
                           ("Emin", "<i4"), ("Emax", "<i4"), ("step", "<u4"), ("n_replicas", "<u4"),
                           ("overlap", "<f8"), ("proposal_kind", "<i4"), ("pad", "<i4")])
assert PA_STATS_DTYPE.itemsize == C.sizeof(PaStats)

_lock = threading.Lock()
_lib = None


def load():
    """Load libgbmc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgbmc.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        lib = C.CDLL(LIB_PATH)
        p, st = C.c_void_p, C.c_int
        sig = {
            "gbmc_version": ([], C.c_int),
            "gbmc_checked_build": ([], C.c_int32),
            "gbmc_last_error": ([], C.c_char_p),
            "gbmc_create": ([C.POINTER(C.c_void_p), C.c_int, p], st),
            "gbmc_set_stream": ([p, p], st),
            "gbmc_sync": ([p], st),
            "gbmc_destroy": ([p], st),
            "gbmc_profile": ([p, C.c_int32], st),
            "gbmc_set_resample_mode": ([p, C.c_int32], st),
            "gbmc_set_sweep_launch": ([p, C.c_int32], st),
            "gbmc_set_sweep_kernel": ([p, C.c_int32], st),
            "pa_state_bytes": ([p, C.POINTER(C.c_size_t)], st),
            "pa_state_save": ([p, p, p, C.c_size_t], st),
            "pa_state_load": ([p, p, p, C.c_size_t], st),
            "gbmc_test_barrier_wait": ([p, C.c_uint32, C.c_uint64], st),
            "gbmc_profile_read": ([p, p, C.c_uint32, C.POINTER(C.c_uint32)], st),
            "gbmc_kernel_launches": ([], C.c_uint64),
            "lattice_init": ([p, C.POINTER(LatticeDesc), p, C.c_size_t, C.POINTER(C.c_void_p)], st),
            "lattice_free": ([p], st),
            "lattice_info": ([p, C.POINTER(LatticeInfo)], st),
            "lattice_set_sweep_counter": ([p, C.c_uint32], st),
            "lattice_copy_out": ([p, p, p, C.c_size_t], st),
            "lattice_copy_in": ([p, p, p, C.c_size_t], st),
            "lattice_couplings_out": ([p, p, p, C.c_size_t], st),
            "metropolis_sweeps": ([p, p, C.c_double, C.c_uint32, p, p], st),
            "metropolis_sweeps_dcb": ([p, p, C.c_double, C.c_uint32, C.c_uint32, C.c_uint32, p, p], st),
            "metropolis_sweeps_msc": ([p, p, C.c_double, C.c_uint32], st),
            "swendsen_wang": ([p, p, C.c_double, C.c_uint32, p, p, p], st),
            "observables": ([p, p, p, p], st),
            "gbmc_autotune": ([p, p, C.c_double, C.c_uint32, C.POINTER(Tuning)], st),
            "gbmc_set_tuning": ([C.c_int32, C.c_int32, C.c_int32, C.POINTER(Tuning)], st),
            "pa_schedule_log": ([p, C.c_uint32, p, C.c_uint32, C.POINTER(C.c_uint32)], st),
            "pa_betas": ([p, C.c_uint32, p, C.c_uint32, C.POINTER(C.c_uint32)], st),
            "gbmc_mlp_param_count": ([], C.c_uint32),
            "mlp_forward": ([p, p, p, C.c_uint32, p], st),
            "mlp_grad": ([p, p, p, p, C.c_uint32, p, p], st),
            "mlp_adam": ([p, p, p, p, p, C.c_uint32, C.c_float], st),
            "mlp_train": ([p, p, p, p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_float, p], st),
            "pt_create": ([p, p, p, C.c_uint32, C.POINTER(C.c_void_p)], st),
            "pt_step": ([p, p, C.c_uint32], st),
            "pt_state_out": ([p, p, p, p, p], st),
            "pt_free": ([p], st),
            "pa_resample_static": ([p, C.c_int32, C.c_int32, C.c_int64, C.c_uint32, C.c_uint32, C.c_uint32,
                                    C.c_uint64, C.c_uint32, C.c_double, p, p, p], st),
            "pa_create": ([p, C.POINTER(C.c_void_p), C.c_uint32, C.POINTER(PaConfig), C.POINTER(C.c_void_p)], st),
            "pa_free": ([p], st),
            "pa_reset": ([p, p, C.c_int32, C.c_uint64], st),
            "pa_populations": ([p, C.POINTER(C.c_uint32)], st),
            "pa_step": ([p, p, p, p], st),
            "pa_run": ([p, p, p, C.c_uint32, C.POINTER(C.c_uint32)], st),
            "pa_run_graph": ([p, p, p, C.c_uint32, C.POINTER(C.c_uint32)], st),
            "pa_parents_out": ([p, p, C.c_uint32, p, C.c_size_t], st),
            "pa_energies_out": ([p, p, C.c_uint32, p, p, C.c_size_t], st),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(status: int):
    if status != GBMC_OK:
        raise GbmcError(status, load().gbmc_last_error().decode(errors="replace"))


def _ptr(x):
    """Raw address of a torch tensor, numpy array or int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    raise TypeError("unsupported buffer type %r" % type(x))


def _nbytes(x):
    if isinstance(x, np.ndarray):
        return x.nbytes
    return x.numel() * x.element_size()


def gbmc_version() -> int:
    return load().gbmc_version()


def gbmc_create(device: int = 0, stream=None):
    h = C.c_void_p()
    _check(load().gbmc_create(C.byref(h), device, stream))
    return h


def gbmc_set_stream(ctx, stream):
    _check(load().gbmc_set_stream(ctx, stream))


def gbmc_sync(ctx):
    _check(load().gbmc_sync(ctx))


def gbmc_destroy(ctx):
    _check(load().gbmc_destroy(ctx))


def gbmc_set_resample_mode(ctx, fused=True):
    _check(load().gbmc_set_resample_mode(ctx, int(bool(fused))))


def gbmc_set_sweep_launch(ctx, mode=GBMC_LAUNCH_AUTO):
    _check(load().gbmc_set_sweep_launch(ctx, int(mode)))


def gbmc_checked_build() -> bool:
    return bool(load().gbmc_checked_build())


def gbmc_set_sweep_kernel(ctx, kernel=GBMC_KERNEL_AUTO):
    _check(load().gbmc_set_sweep_kernel(ctx, int(kernel)))


def gbmc_test_barrier_wait(ctx, phantom_arrivals=0, budget_cycles=2000000000):
    _check(load().gbmc_test_barrier_wait(ctx, phantom_arrivals, budget_cycles))


def gbmc_profile(ctx, enable=True):
    _check(load().gbmc_profile(ctx, int(bool(enable))))


def gbmc_profile_read(ctx) -> dict:
    """{kernel name: (launches, total_ms)} recorded since gbmc_profile(ctx, True)."""
    arr = (KernelTime * 32)()
    n = C.c_uint32()
    _check(load().gbmc_profile_read(ctx, C.cast(arr, C.c_void_p), 32, C.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n.value)}


def gbmc_kernel_launches() -> int:
    return int(load().gbmc_kernel_launches())


def lattice_init(ctx, dim, L, model=GBMC_ISING_FM, start=GBMC_START_RANDOM, n_instances=1, n_replicas=1,
                 seed=1, instance_base=0, layout=GBMC_INT8, spins=None):
    d = LatticeDesc(dim, L, model, layout, start, n_instances, n_replicas, instance_base, seed)
    h = C.c_void_p()
    _check(load().lattice_init(ctx, C.byref(d), _ptr(spins), 0 if spins is None else _nbytes(spins), C.byref(h)))
    return h


def lattice_free(lat):
    _check(load().lattice_free(lat))


def lattice_info(lat) -> LatticeInfo:
    info = LatticeInfo()
    _check(load().lattice_info(lat, C.byref(info)))
    return info


def lattice_set_sweep_counter(lat, t: int):
    _check(load().lattice_set_sweep_counter(lat, t))


def lattice_copy_out(ctx, lat, dst):
    _check(load().lattice_copy_out(ctx, lat, _ptr(dst), _nbytes(dst)))
    return dst


def lattice_copy_in(ctx, lat, src):
    _check(load().lattice_copy_in(ctx, lat, _ptr(src), _nbytes(src)))


def lattice_couplings_out(ctx, lat, dst):
    _check(load().lattice_couplings_out(ctx, lat, _ptr(dst), _nbytes(dst)))
    return dst


def metropolis_sweeps(ctx, lat, beta: float, n_sweeps: int, E_series=None, M_series=None):
    _check(load().metropolis_sweeps(ctx, lat, float(beta), n_sweeps, _ptr(E_series), _ptr(M_series)))


def metropolis_sweeps_dcb(ctx, lat, beta: float, n_rounds: int, k: int, tile: int = 64, E_series=None,
                          M_series=None):
    _check(load().metropolis_sweeps_dcb(ctx, lat, float(beta), n_rounds, k, tile, _ptr(E_series),
                                        _ptr(M_series)))


def metropolis_sweeps_msc(ctx, lat, beta: float, n_sweeps: int):
    _check(load().metropolis_sweeps_msc(ctx, lat, float(beta), n_sweeps))


def swendsen_wang(ctx, lat, beta: float, n_updates: int, E_series=None, M_series=None, labels=None):
    _check(load().swendsen_wang(ctx, lat, float(beta), n_updates, _ptr(E_series), _ptr(M_series), _ptr(labels)))


def observables(ctx, lat, E=None, M=None):
    _check(load().observables(ctx, lat, _ptr(E), _ptr(M)))


def gbmc_autotune(ctx, lat, beta, n_sweeps=10) -> Tuning:
    t = Tuning()
    _check(load().gbmc_autotune(ctx, lat, float(beta), n_sweeps, C.byref(t)))
    return t


def gbmc_set_tuning(dim, model, L, threads_per_copy=None, copies_per_cta=1, row_walk=True, persistent=False,
                    kernel=GBMC_KERNEL_BYTES):
    """Force a launch shape for a lattice class; threads_per_copy=None clears it."""
    if threads_per_copy is None:
        _check(load().gbmc_set_tuning(dim, model, L, None))
        return
    t = Tuning(1, threads_per_copy, copies_per_cta, int(bool(row_walk)), 0.0, 0, int(bool(persistent)), int(kernel))
    _check(load().gbmc_set_tuning(dim, model, L, C.byref(t)))


def pa_create(ctx, lattices, theta, n_steps, schedule=GBMC_SCHED_LINEAR, beta_f=1.0, betas=None, init=True,
              target_overlap=0.85, dbeta_max=0.05, mlp_params=None, overlap_lo=0.83, overlap_hi=0.90,
              resample=GBMC_RESAMPLE_MULTINOMIAL, initial_replicas=0, sweep_rng=GBMC_RNG_PHILOX):
    arr = (C.c_void_p * len(lattices))(*[l.value if isinstance(l, C.c_void_p) else l for l in lattices])
    keep = []
    bptr = None
    if betas is not None:
        b = np.ascontiguousarray(betas, dtype=np.float64)
        keep.append(b)
        bptr = b.ctypes.data
    mptr = None
    if mlp_params is not None:
        m = np.ascontiguousarray(mlp_params, dtype=np.float32)
        keep.append(m)
        mptr = m.ctypes.data
    cfg = PaConfig(theta, n_steps, schedule, int(bool(init)), beta_f, bptr, target_overlap, dbeta_max, mptr,
                   overlap_lo, overlap_hi, resample, initial_replicas, sweep_rng, 0)
    h = C.c_void_p()
    _check(load().pa_create(ctx, arr, len(lattices), C.byref(cfg), C.byref(h)))
    return h


def pa_free(pa):
    _check(load().pa_free(pa))


def pa_reset(ctx, pa, init=True, seed=0):
    _check(load().pa_reset(ctx, pa, int(bool(init)), seed))


def pa_populations(pa) -> int:
    n = C.c_uint32()
    _check(load().pa_populations(pa, C.byref(n)))
    return n.value


def pa_step(ctx, pa, beta_next=None, want_stats=True):
    out = None
    if want_stats:
        out = np.zeros(pa_populations(pa), dtype=PA_STATS_DTYPE)
    bn = None
    if beta_next is not None:
        bn = np.ascontiguousarray(beta_next, dtype=np.float64)
    _check(load().pa_step(ctx, pa, _ptr(bn), _ptr(out)))
    return out


def pa_run(ctx, pa, capacity=None):
    P = pa_populations(pa)
    out = None
    cap = 0
    if capacity is not None:
        cap = capacity
        out = np.zeros((capacity, P), dtype=PA_STATS_DTYPE)
    n = C.c_uint32()
    _check(load().pa_run(ctx, pa, _ptr(out), cap, C.byref(n)))
    return (out[: n.value + 1] if out is not None else None), n.value


def pa_run_graph(ctx, pa, capacity=None):
    P = pa_populations(pa)
    out = None
    cap = 0
    if capacity is not None:
        cap = capacity
        out = np.zeros((capacity, P), dtype=PA_STATS_DTYPE)
    n = C.c_uint32()
    _check(load().pa_run_graph(ctx, pa, _ptr(out), cap, C.byref(n)))
    return (out[: n.value + 1] if out is not None else None), n.value


def pa_parents_out(ctx, pa, lattice, dst):
    _check(load().pa_parents_out(ctx, pa, lattice, _ptr(dst), dst.size if isinstance(dst, np.ndarray) else dst.numel()))
    return dst


def pa_energies_out(ctx, pa, lattice, E_dst=None, M_dst=None):
    ref = E_dst if E_dst is not None else M_dst
    n = ref.size if isinstance(ref, np.ndarray) else ref.numel()
    _check(load().pa_energies_out(ctx, pa, lattice, _ptr(E_dst), _ptr(M_dst), n))


def gbmc_last_error() -> str:
    return load().gbmc_last_error().decode(errors="replace")


def pa_resample_static(stream, device, dim, n_sites, n_instances, n_replicas, instance_base, seed, step, dbeta,
                       E, parent, lnQ):
    """Allocation-free resampling step (static device scratch); see include/gbmc.h."""
    _check(load().pa_resample_static(stream, device, dim, n_sites, n_instances, n_replicas, instance_base, seed,
                                     step, float(dbeta), _ptr(E), _ptr(parent), _ptr(lnQ)))


def pa_schedule_log(pa, lattice=0) -> list:
    """Per-step records of an adaptive schedule (dicts)."""
    n = C.c_uint32()
    _check(load().pa_schedule_log(pa, lattice, None, 0, C.byref(n)))
    arr = (ScheduleRecord * max(1, n.value))()
    _check(load().pa_schedule_log(pa, lattice, C.cast(arr, C.c_void_p), n.value, C.byref(n)))
    out = []
    for i in range(n.value):
        r = arr[i]
        out.append({k: (list(getattr(r, k)) if k == "features" else getattr(r, k))
                    for k, _ in ScheduleRecord._fields_ if k != "pad"})
    return out


def pa_state_bytes(pa) -> int:
    n = C.c_size_t()
    _check(load().pa_state_bytes(pa, C.byref(n)))
    return n.value


def pa_state_save(ctx, pa) -> np.ndarray:
    """The run's state between steps as a byte array (spins not included)."""
    buf = np.zeros(pa_state_bytes(pa), dtype=np.uint8)
    _check(load().pa_state_save(ctx, pa, _ptr(buf), buf.nbytes))
    return buf


def pa_state_load(ctx, pa, state):
    buf = np.ascontiguousarray(state, dtype=np.uint8)
    _check(load().pa_state_load(ctx, pa, _ptr(buf), buf.nbytes))


def pa_betas(pa, lattice=0) -> np.ndarray:
    n = C.c_uint32()
    _check(load().pa_betas(pa, lattice, None, 0, C.byref(n)))
    out = np.zeros(n.value, dtype=np.float64)
    _check(load().pa_betas(pa, lattice, _ptr(out), n.value, C.byref(n)))
    return out


def gbmc_mlp_param_count() -> int:
    return int(load().gbmc_mlp_param_count())


def mlp_forward(ctx, params, X, Y):
    _check(load().mlp_forward(ctx, _ptr(params), _ptr(X), X.shape[0], _ptr(Y)))


def mlp_grad(ctx, params, X, T, grad, loss):
    _check(load().mlp_grad(ctx, _ptr(params), _ptr(X), _ptr(T), X.shape[0], _ptr(grad), _ptr(loss)))


def mlp_adam(ctx, params, grad, m, v, k, lr):
    _check(load().mlp_adam(ctx, _ptr(params), _ptr(grad), _ptr(m), _ptr(v), k, float(lr)))


def mlp_train(ctx, params, X, T, epochs, batch, lr, loss_out=None):
    _check(load().mlp_train(ctx, _ptr(params), _ptr(X), _ptr(T), X.shape[0], epochs, batch, float(lr),
                            _ptr(loss_out)))


def pt_create(ctx, lat, betas, theta):
    b = np.ascontiguousarray(betas, dtype=np.float64)
    h = C.c_void_p()
    _check(load().pt_create(ctx, lat, b.ctypes.data, theta, C.byref(h)))
    return h


def pt_step(ctx, pt, n_steps=1):
    _check(load().pt_step(ctx, pt, n_steps))


def pt_state_out(ctx, pt, rep_of=None, accepted=None, E=None):
    _check(load().pt_state_out(ctx, pt, _ptr(rep_of), _ptr(accepted), _ptr(E)))


def pt_free(pt):
    _check(load().pt_free(pt))
