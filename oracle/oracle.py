"""ctypes wrapper of the CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module.  The product path (the CUDA
library under ``paper_2501_17267_gb300``) never imports it.

The oracle is a plain, sequential restatement of arXiv:2501.17267's spin-glass
setting: Eq. 1 (energy), Eq. 2 (optimality gap), the tile-planting instances of
Sec. II, Metropolis simulated annealing (App. D.1) and parallel tempering
(App. D.2).  All arrays are numpy; spins are int8 in {-1, +1}; couplings J3 are
int8 with shape (N, 3), N = L^3, entry [i, d] being the coupling on the edge from
site i = x + L*(y + L*z) to its +1 neighbour along axis d.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CLASS_F22, CLASS_F42, CLASS_F6 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with plain gcc (no fast-math, no FMA contraction)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
             "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64, u32, u64, dbl = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint32,
                                       ctypes.c_uint64, ctypes.c_double)
            sig = {
                "or_philox4x32_10": (None, [P, P, P]),
                "or_site": (i64, [i32, i32, i32, i32]),
                "or_energy": (i64, [i32, P, P]),
                "or_local_field": (i32, [i32, P, P, i64]),
                "or_epsilon": (dbl, [i64, i64]),
                "or_cube_edge": (None, [i32, P, P]),
                "or_tile_template": (i32, [i32, P]),
                "or_tile_energy": (i32, [P, i32]),
                "or_tile_bruteforce": (None, [P, P, P]),
                "or_cube_symmetry": (i32, [i32, i32]),
                "or_generate": (i32, [i32, u64, P, i32, P, P, P]),
                "or_beta_schedule": (None, [i32, dbl, dbl, i32, P]),
                "or_pt_ladder": (None, [i32, dbl, dbl, P]),
                "or_metropolis_threshold": (u32, [dbl, i32]),
                "or_exchange_threshold": (u32, [dbl, i64]),
                "or_init_spin": (ctypes.c_int8, [u64, u32, i64, i32]),
                "or_metropolis_uniform_grid": (None, [u64, u32, i64, i32, u32, i32, P, i32, P]),
                "or_sa_run": (i32, [i32, P, u64, u32, i32, dbl, dbl, i32, P, i32, P, P]),
                "or_pt_run": (i32, [i32, P, u64, u32, i32, i32, dbl, dbl, P, P, P, P, P]),
                "or_fragment_run": (i32, [i32, P, i32, i32, dbl, dbl, u64, u32, P, P]),
                "or_fragment_min_energies": (i32, [i32, P, P, i32, P, P]),
                "or_fragment_tropical": (i32, [i32, P, i32, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def site(L: int, x: int, y: int, z: int) -> int:
    return int(lib().or_site(L, x, y, z))


def energy(L: int, J3: np.ndarray, s: np.ndarray) -> int:
    J3 = np.ascontiguousarray(J3, dtype=np.int8)
    s = np.ascontiguousarray(s, dtype=np.int8)
    assert J3.size == 3 * L ** 3 and s.size == L ** 3
    return int(lib().or_energy(L, _p(J3), _p(s)))


def local_field(L: int, J3: np.ndarray, s: np.ndarray, i: int) -> int:
    J3 = np.ascontiguousarray(J3, dtype=np.int8)
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(lib().or_local_field(L, _p(J3), _p(s), i))


def epsilon(E: int, E_gs: int) -> float:
    return float(lib().or_epsilon(int(E), int(E_gs)))


def cube_edge(e: int):
    u, v = ctypes.c_int(), ctypes.c_int()
    lib().or_cube_edge(e, ctypes.byref(u), ctypes.byref(v))
    return u.value, v.value


def tile_template(cls: int) -> np.ndarray:
    J = np.zeros(12, dtype=np.int8)
    if lib().or_tile_template(cls, _p(J)) != 0:
        raise ValueError(cls)
    return J


def tile_energy(J12: np.ndarray, state: int) -> int:
    J12 = np.ascontiguousarray(J12, dtype=np.int8)
    return int(lib().or_tile_energy(_p(J12), state))


def tile_bruteforce(J12: np.ndarray):
    J12 = np.ascontiguousarray(J12, dtype=np.int8)
    emin, deg = ctypes.c_int(), ctypes.c_int()
    lib().or_tile_bruteforce(_p(J12), ctypes.byref(emin), ctypes.byref(deg))
    return emin.value, deg.value


def cube_symmetry(sym: int, corner: int) -> int:
    return int(lib().or_cube_symmetry(sym, corner))


def generate(L: int, seed: int, class_prob=(1 / 3, 1 / 3, 1 / 3), gauge: bool = True):
    """Tile-planted instance -> (J3 int8 (N,3), planted tau int8 (N,), E_gs int)."""
    N = L ** 3
    J3 = np.zeros((N, 3), dtype=np.int8)
    tau = np.zeros(N, dtype=np.int8)
    cp = np.ascontiguousarray(class_prob, dtype=np.float64)
    egs = ctypes.c_int64()
    rc = lib().or_generate(L, seed, _p(cp), int(bool(gauge)), _p(J3), _p(tau), ctypes.byref(egs))
    if rc != 0:
        raise ValueError(f"or_generate failed ({rc})")
    return J3, tau, int(egs.value)


def beta_schedule(S: int, b0: float, b1: float, geometric: bool = False) -> np.ndarray:
    out = np.zeros(max(S, 1), dtype=np.float64)
    lib().or_beta_schedule(S, b0, b1, int(bool(geometric)), _p(out))
    return out[:S]


def pt_ladder(K: int, bmin: float, bmax: float) -> np.ndarray:
    out = np.zeros(K, dtype=np.float64)
    lib().or_pt_ladder(K, bmin, bmax, _p(out))
    return out


def metropolis_threshold(beta: float, dE: int) -> int:
    return int(lib().or_metropolis_threshold(beta, dE))


def exchange_threshold(dbeta: float, d: int) -> int:
    return int(lib().or_exchange_threshold(dbeta, d))


def init_spin(seed: int, instance_id: int, i: int, rep: int) -> int:
    return int(lib().or_init_spin(seed, instance_id, i, rep))


def metropolis_uniforms(seed: int, instance_id: int, i0: int, n_sites: int, s0: int, n_sweeps: int,
                        reps) -> np.ndarray:
    """The 32-bit draws U of the listed replicas at sites i0.. and sweeps s0..:
    uint32 array (n_sweeps, n_sites, len(reps))."""
    reps = np.ascontiguousarray(list(reps), dtype=np.int32)
    out = np.zeros((n_sweeps, n_sites, len(reps)), dtype=np.uint32)
    lib().or_metropolis_uniform_grid(seed, instance_id, i0, n_sites, s0, n_sweeps, _p(reps), len(reps), _p(out))
    return out


def sa_run(L: int, J3: np.ndarray, seed: int, instance_id: int, S: int, b0: float,
           b1: float, geometric: bool = False, reps=None, R: int | None = None):
    """Simulated annealing of the listed replicas.  -> (spins int8 (n, N), E int64 (n,))."""
    if reps is None:
        reps = range(R)
    reps = np.ascontiguousarray(list(reps), dtype=np.int32)
    N = L ** 3
    J3 = np.ascontiguousarray(J3, dtype=np.int8)
    spins = np.zeros((len(reps), N), dtype=np.int8)
    E = np.zeros(len(reps), dtype=np.int64)
    rc = lib().or_sa_run(L, _p(J3), seed, instance_id, S, b0, b1, int(bool(geometric)),
                         _p(reps), len(reps), _p(spins), _p(E))
    if rc != 0:
        raise ValueError(f"or_sa_run failed ({rc})")
    return spins, E


def pt_run(L: int, J3: np.ndarray, seed: int, instance_id: int, K: int, S: int,
           bmin: float, bmax: float):
    """Parallel tempering.  -> dict(spins (K,N) by slot, E (K,), perm (K,) slot->rung,
    minE, accepts (K-1,))."""
    N = L ** 3
    J3 = np.ascontiguousarray(J3, dtype=np.int8)
    spins = np.zeros((K, N), dtype=np.int8)
    E = np.zeros(K, dtype=np.int64)
    perm = np.zeros(K, dtype=np.int32)
    acc = np.zeros(max(K - 1, 1), dtype=np.int64)
    minE = ctypes.c_int64()
    rc = lib().or_pt_run(L, _p(J3), seed, instance_id, K, S, bmin, bmax, _p(spins), _p(E),
                         _p(perm), ctypes.byref(minE), _p(acc))
    if rc != 0:
        raise ValueError(f"or_pt_run failed ({rc})")
    return {"spins": spins, "E": E, "perm": perm, "minE": int(minE.value),
            "accepts": acc[: max(K - 1, 0)]}


def fragment_run(L: int, J3: np.ndarray, l: int, S: int, b0: float, b1: float, seed: int = 0,
                 instance_id: int = 0):
    """Fragment meta-heuristic with SA fragment anneals (Sec. II, App. A; see
    or_fragment_run).  -> (spins (N,) int8, E)."""
    N = L ** 3
    J3 = np.ascontiguousarray(J3, dtype=np.int8)
    spins = np.zeros(N, dtype=np.int8)
    E = ctypes.c_int64()
    rc = lib().or_fragment_run(L, _p(J3), l, S, b0, b1, seed, instance_id, _p(spins), ctypes.byref(E))
    if rc != 0:
        raise ValueError(f"or_fragment_run failed ({rc})")
    return spins, int(E.value)


def fragment_min_energies(h, Jff, c: int):
    """Lowest energy of sum_k h_k s_k + sum_{k<j} Jff[k, j] s_k s_j over the states with
    s_c = +1 and with s_c = -1 (exact enumeration).  -> (m_plus, m_minus)."""
    h = np.ascontiguousarray(h, dtype=np.int32)
    J = np.ascontiguousarray(Jff, dtype=np.int8)
    mp, mm = ctypes.c_int64(), ctypes.c_int64()
    rc = lib().or_fragment_min_energies(len(h), _p(h), _p(J), c, ctypes.byref(mp), ctypes.byref(mm))
    if rc != 0:
        raise ValueError(f"or_fragment_min_energies failed ({rc})")
    return int(mp.value), int(mm.value)


def fragment_tropical(L: int, J3: np.ndarray, l: int):
    """Fragment decimation with exact zero-temperature fragment marginals (l <= 3).
    -> (spins (N,) int8, E)."""
    J3 = np.ascontiguousarray(J3, dtype=np.int8)
    spins = np.zeros(L ** 3, dtype=np.int8)
    E = ctypes.c_int64()
    rc = lib().or_fragment_tropical(L, _p(J3), l, _p(spins), ctypes.byref(E))
    if rc != 0:
        raise ValueError(f"or_fragment_tropical failed ({rc})")
    return spins, int(E.value)
