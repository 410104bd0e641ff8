"""CPU oracle for checkerboard Metropolis and population annealing.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. It shares no code with the CUDA library (``paper_1709_04394_gb300``)
and never imports it.

The arithmetic lives in ``gbmc_oracle.c`` (plain C, one site at a time, in the
order of the paper's algorithms; see that file's header for the passages it
follows and the readings it takes). This module compiles it with the host C
compiler on first use and marshals numpy arrays through ctypes. The schedule
helpers of Sec. 5.4 that the paper leaves open (histogram overlap, bisection)
live in ``schedule.py``; the MLP reference lives in ``mlp.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gbmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

PURPOSE_METRO, PURPOSE_INIT, PURPOSE_RESAMPLE, PURPOSE_COUPLING = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile gbmc_oracle.c into _build/liboracle.so (host C compiler, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        p = C.c_void_p
        u32, u64, i32, i64, dbl = C.c_uint32, C.c_uint64, C.c_int, C.c_int64, C.c_double
        lib.orc_philox_batch.argtypes = [i64, p, p, p]
        lib.orc_thresholds.argtypes = [dbl, i32, p]
        lib.orc_init_spins.argtypes = [i32, i32, u64, u32, u32, i32, p]
        lib.orc_couplings.argtypes = [i32, u64, u32, p]
        lib.orc_halfsweep.argtypes = [i32, i32, p, p, p, u64, u32, u32, u32, i32]
        lib.orc_sweeps.argtypes = [i32, i32, p, p, dbl, u64, u32, u32, u32, u32]
        lib.orc_dcb_sweeps.argtypes = [i32, i32, p, dbl, u64, u32, u32, u32, u32, u32]
        lib.orc_observables.argtypes = [i32, i32, p, p, p, p]
        lib.orc_resample.argtypes = [u32, p, dbl, u64, u32, u32, p]
        lib.orc_resample.restype = dbl
        lib.orc_resample_nearest.argtypes = [u32, p, dbl, u32, u32, u64, u32, u32, p, p]
        lib.orc_resample_nearest.restype = dbl
        lib.orc_pa_run_nearest.argtypes = [i32, i32, p, u64, u32, u32, u32, u32, p, u32, p, i32,
                                           p, p, p, p, p, p, i32, i32]
        lib.orc_exp_neg.argtypes = [dbl]
        lib.orc_exp_neg.restype = dbl
        lib.orc_poisson.argtypes = [dbl, u64]
        lib.orc_poisson.restype = u32
        lib.orc_resample_poisson.argtypes = [u32, p, dbl, u32, u32, u64, u32, u32, p, p]
        lib.orc_resample_poisson.restype = dbl
        lib.orc_pa_run_nearest.restype = i32
        lib.orc_children_order.argtypes = [u32, p, p]
        lib.orc_pt_run.argtypes = [i32, i32, p, u64, u32, u32, p, u32, u32, u32, u32, p, p, p, p]
        lib.orc_pa_run.argtypes = [i32, i32, p, u64, u32, u32, u32, p, u32, p, i32,
                                   p, p, p, p, p, p, p, p, p, p, p, i32]
        lib.orc_msc_sweeps.argtypes = [i32, i32, p, p, dbl, u64, u32, u32, u32, u32]
        lib.orc_msc_uniforms.argtypes = [u64, u64, u32, u32, i32, u32, p]
        lib.orc_sw_bond_threshold.argtypes = [dbl]
        lib.orc_sw_bond_threshold.restype = C.c_int64
        lib.orc_sw_update.argtypes = [i32, i32, p, dbl, u64, u32, u32, u32, p]
        lib.orc_sw_bonds.argtypes = [i32, i32, p, dbl, u64, u32, u32, u32, p]
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of counters ``ctr`` (shape [n,4] uint32) under ``key`` (2 uint32)."""
    lib = _load()
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(ctr)
    lib.orc_philox_batch(ctr.shape[0], _ptr(ctr), _ptr(key), _ptr(out))
    return out


def thresholds(beta: float, ndE: int) -> np.ndarray:
    """int64 T(4), T(8), ... : accept a positive dE iff the 32-bit word u <= T(dE)."""
    lib = _load()
    out = np.empty(ndE, dtype=np.int64)
    lib.orc_thresholds(float(beta), ndE, _ptr(out))
    return out


def n_sites(dim: int, L: int) -> int:
    return L ** dim


def init_spins(dim: int, L: int, seed: int, instance: int, replica: int, random_start: bool) -> np.ndarray:
    lib = _load()
    s = np.empty(n_sites(dim, L), dtype=np.int8)
    lib.orc_init_spins(dim, L, seed, instance, replica, int(bool(random_start)), _ptr(s))
    return s


def couplings(L: int, seed: int, instance: int) -> np.ndarray:
    """Bimodal couplings of a dim-3 lattice, int8 [N, 3] (forward x, y, z bonds)."""
    lib = _load()
    J = np.empty(n_sites(3, L) * 3, dtype=np.int8)
    lib.orc_couplings(L, seed, instance, _ptr(J))
    return J.reshape(-1, 3)


def _check_spins(s, dim, L):
    assert s.dtype == np.int8 and s.flags.c_contiguous and s.size == n_sites(dim, L)


def halfsweep(dim, L, s, J, thr, seed, instance, replica, t, colour):
    lib = _load()
    _check_spins(s, dim, L)
    thr = np.ascontiguousarray(thr, dtype=np.int64)
    Jc = None if J is None else np.ascontiguousarray(J, dtype=np.int8)
    lib.orc_halfsweep(dim, L, _ptr(s), _ptr(Jc), _ptr(thr), seed, instance, replica, t, colour)


def sweeps(dim, L, s, J, beta, seed, instance, replica, t0, n):
    """n checkerboard sweeps of spins ``s`` (int8, in place) at ``beta``."""
    lib = _load()
    _check_spins(s, dim, L)
    Jc = None if J is None else np.ascontiguousarray(J, dtype=np.int8)
    lib.orc_sweeps(dim, L, _ptr(s), _ptr(Jc), float(beta), seed, instance, replica, t0, n)


def msc_uniforms(seed, k, t, group, colour, instance):
    """The 32 uniforms of replicas 32 group .. 32 group + 31 at colour-rank k."""
    lib = _load()
    out = np.empty(32, dtype=np.uint32)
    lib.orc_msc_uniforms(seed, k, t, group, colour, instance, _ptr(out))
    return out


def msc_sweeps(dim, L, s, J, beta, seed, instance, replica, t0, n):
    """n checkerboard sweeps of replica ``replica`` with the multi-spin-coded
    random numbers (reading R18): LCG outputs seeded per 32-replica group."""
    lib = _load()
    _check_spins(s, dim, L)
    Jc = None if J is None else np.ascontiguousarray(J, dtype=np.int8)
    lib.orc_msc_sweeps(dim, L, _ptr(s), _ptr(Jc), float(beta), seed, instance, replica, t0, n)


def sw_bond_threshold(beta):
    """T_bond = ceil((1 - exp(-2 beta)) 2^32) - 1 of the Swendsen-Wang bonds."""
    return int(_load().orc_sw_bond_threshold(float(beta)))


def sw_bonds(dim, L, s, beta, seed, instance, replica, t):
    """Active flags [N, dim] of the forward bonds in a Swendsen-Wang update."""
    lib = _load()
    _check_spins(s, dim, L)
    a = np.empty(s.size * dim, dtype=np.uint8)
    lib.orc_sw_bonds(dim, L, _ptr(np.ascontiguousarray(s)), float(beta), seed, instance, replica, t, _ptr(a))
    return a.reshape(s.size, dim)


def sw_update(dim, L, s, beta, seed, instance, replica, t, want_labels=False):
    """One Swendsen-Wang update (Sec. 3.3; reading R19) of ferromagnet ``s``
    (int8, in place) with counter t; optionally returns the cluster name
    (smallest site index) of every site before the flip."""
    lib = _load()
    _check_spins(s, dim, L)
    lab = np.empty(s.size, dtype=np.int32) if want_labels else None
    lib.orc_sw_update(dim, L, _ptr(s), float(beta), seed, instance, replica, t, _ptr(lab))
    return lab


def dcb_sweeps(L, tile, s, beta, seed, instance, replica, t0, k, n_rounds):
    """n_rounds double-checkerboard rounds (k sweeps per tile and round) of a
    2D ferromagnet ``s`` (int8, in place); the sweep counter advances by k
    per round."""
    lib = _load()
    _check_spins(s, 2, L)
    if tile <= 0 or tile % 2 or L % (2 * tile):
        raise ValueError("L must be a multiple of 2 * tile")
    lib.orc_dcb_sweeps(L, tile, _ptr(s), float(beta), seed, instance, replica, t0, k, n_rounds)


def observables(dim, L, s, J=None):
    lib = _load()
    _check_spins(s, dim, L)
    Jc = None if J is None else np.ascontiguousarray(J, dtype=np.int8)
    E = np.zeros(1, dtype=np.int64)
    M = np.zeros(1, dtype=np.int64)
    lib.orc_observables(dim, L, _ptr(s), _ptr(Jc), _ptr(E), _ptr(M))
    return int(E[0]), int(M[0])


def resample(E, dbeta, seed, instance, step):
    """Multinomial resampling counts and ln Q of one annealing step."""
    lib = _load()
    E = np.ascontiguousarray(E, dtype=np.int64)
    counts = np.empty(E.size, dtype=np.uint32)
    lnQ = lib.orc_resample(E.size, _ptr(E), float(dbeta), seed, instance, step, _ptr(counts))
    return counts, lnQ


def resample_nearest(E, dbeta, R0, cap, seed, instance, step):
    """Nearest-integer resampling counts (variable population), the new
    population size and ln Q of one annealing step (reading R17)."""
    lib = _load()
    E = np.ascontiguousarray(E, dtype=np.int64)
    counts = np.empty(E.size, dtype=np.uint32)
    Rn = np.zeros(1, dtype=np.uint64)
    lnQ = lib.orc_resample_nearest(E.size, _ptr(E), float(dbeta), R0, cap, seed, instance, step, _ptr(counts),
                                   _ptr(Rn))
    return counts, int(Rn[0]), lnQ


def children_order(counts):
    """Slot -> parent map: children of parent j contiguous, parents in order."""
    lib = _load()
    counts = np.ascontiguousarray(counts, dtype=np.uint32)
    parent = np.empty(int(counts.sum(dtype=np.uint64)), dtype=np.uint32)
    lib.orc_children_order(counts.size, _ptr(counts), _ptr(parent))
    return parent


def linear_betas(beta_f: float, S: int) -> np.ndarray:
    """beta_i = (beta_f * i) / S, i = 0..S, evaluated in that order in fp64."""
    return np.array([(float(beta_f) * float(i)) / float(S) for i in range(S + 1)], dtype=np.float64)


def pa_run(dim, L, seed, instance, R, betas, theta, J=None, spins=None, keep_energies=False, msc=False):
    """Population annealing for one instance (Sec. 5.4). Returns a dict of per-step
    arrays (index 0 = beta_0 = 0) and the final population. msc: sweeps with the
    multi-spin-coded random numbers (reading R18)."""
    lib = _load()
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    S = betas.size - 1
    N = n_sites(dim, L)
    init = spins is None
    if init:
        spins = np.empty(R * N, dtype=np.int8)
    else:
        spins = np.ascontiguousarray(spins, dtype=np.int8).reshape(-1).copy()
        assert spins.size == R * N
    Jc = None if J is None else np.ascontiguousarray(J, dtype=np.int8)
    out = {k: np.zeros(S + 1, dtype=np.float64) for k in ("lnQ", "lnZ", "sumE2", "sumM2")}
    sumE = np.zeros(S + 1, dtype=np.int64)
    sumAbsM = np.zeros(S + 1, dtype=np.int64)
    hashes = np.zeros(S + 1, dtype=np.uint64)
    E = np.zeros(R, dtype=np.int64)
    M = np.zeros(R, dtype=np.int64)
    parents = np.arange(R, dtype=np.uint32)
    E_steps = np.zeros((S + 1, R), dtype=np.int64) if keep_energies else None
    lib.orc_pa_run(dim, L, _ptr(Jc), seed, instance, R, S, _ptr(betas), theta, _ptr(spins),
                   int(init), _ptr(out["lnQ"]), _ptr(out["lnZ"]), _ptr(sumE), _ptr(out["sumE2"]),
                   _ptr(sumAbsM), _ptr(out["sumM2"]), _ptr(hashes), _ptr(E), _ptr(M), _ptr(parents),
                   _ptr(E_steps), int(bool(msc)))
    out.update(sumE=sumE, sumAbsM=sumAbsM, counts_hash=hashes, E=E, M=M, parents=parents, E_steps=E_steps,
               spins=spins.reshape(R, N), betas=betas)
    return out


def exp_neg(x):
    """e^{-x} of reading R20 (IEEE-exact sequence, not libm)."""
    return float(_load().orc_exp_neg(float(x)))


def poisson(tau, U64):
    """Poisson(tau) count by inversion from the 64-bit uniform U64 (reading R20)."""
    return int(_load().orc_poisson(float(tau), int(U64)))


def resample_poisson(E, dbeta, R0, cap, seed, instance, step):
    """Poisson resampling counts (variable population), the new population size
    and ln Q of one annealing step (reading R20)."""
    lib = _load()
    E = np.ascontiguousarray(E, dtype=np.int64)
    counts = np.empty(E.size, dtype=np.uint32)
    Rn = np.zeros(1, dtype=np.uint64)
    lnQ = lib.orc_resample_poisson(E.size, _ptr(E), float(dbeta), R0, cap, seed, instance, step, _ptr(counts),
                                   _ptr(Rn))
    return counts, int(Rn[0]), lnQ


def pa_run_nearest(dim, L, seed, instance, R0, cap, betas, theta, J=None, msc=False, poisson=False):
    """Population annealing with nearest-integer resampling and a variable
    population (at most cap replicas). Returns a dict of per-step arrays
    (lnQ, lnZ, sumE, nrep), the final population (its first nrep[-1] rows)
    and ok = False if a step would have needed more than cap replicas."""
    lib = _load()
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    S = betas.size - 1
    N = n_sites(dim, L)
    spins = np.zeros(cap * N, dtype=np.int8)
    Jc = None if J is None else np.ascontiguousarray(J, dtype=np.int8)
    lnQ = np.zeros(S + 1)
    lnZ = np.zeros(S + 1)
    sumE = np.zeros(S + 1, dtype=np.int64)
    nrep = np.zeros(S + 1, dtype=np.uint32)
    E = np.zeros(cap, dtype=np.int64)
    parents = np.zeros(cap, dtype=np.uint32)
    rc = lib.orc_pa_run_nearest(dim, L, _ptr(Jc), seed, instance, R0, cap, S, _ptr(betas), theta, _ptr(spins), 1,
                                _ptr(lnQ), _ptr(lnZ), _ptr(sumE), _ptr(nrep), _ptr(E), _ptr(parents), int(bool(msc)),
                                int(bool(poisson)))
    n = int(nrep[S]) if rc == 0 else 0
    return dict(lnQ=lnQ, lnZ=lnZ, sumE=sumE, nrep=nrep, ok=rc == 0, spins=spins.reshape(cap, N)[:n],
                E=E[:n], parents=parents[:n], betas=betas)


def pt_run(dim, L, seed, instance, betas, theta, n_steps, J=None, spins=None, rep_of=None, accepted=None,
           t0=0, round0=0):
    """Parallel tempering (Sec. 5.1, Eq. (10)) of len(betas) replicas of one instance.
    Returns (spins [T, N], rep_of [T], accepted [T-1], E [T]) after n_steps steps."""
    lib = _load()
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    T = betas.size
    N = n_sites(dim, L)
    if spins is None:
        spins = np.stack([init_spins(dim, L, seed, instance, r, True) for r in range(T)])
    spins = np.ascontiguousarray(spins, dtype=np.int8).reshape(T, N).copy()
    rep_of = np.arange(T, dtype=np.uint32) if rep_of is None else np.ascontiguousarray(rep_of, dtype=np.uint32).copy()
    accepted = np.zeros(T - 1, dtype=np.uint32) if accepted is None else np.ascontiguousarray(accepted, dtype=np.uint32).copy()
    E = np.zeros(T, dtype=np.int64)
    Jc = None if J is None else np.ascontiguousarray(J, dtype=np.int8)
    lib.orc_pt_run(dim, L, _ptr(Jc), seed, instance, T, _ptr(betas), theta, n_steps, t0, round0, _ptr(spins),
                   _ptr(rep_of), _ptr(accepted), _ptr(E))
    return spins, rep_of, accepted, E
