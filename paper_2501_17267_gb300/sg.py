"""Thin ctypes binding of libsg (C ABI in include/sg.h).

Argument marshalling only: every step of the path runs in the CUDA library.
Host arrays are numpy; device arrays are torch CUDA tensors (PyTorch supplies
device memory and the current stream, nothing else).  Importing this module
loads ``libsg.so`` and raises if it has not been built -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsg.so")

SG_OK, SG_EINVAL, SG_ENOMEM, SG_ECUDA, SG_ETIMEOUT, SG_EBUSY, SG_EINTERNAL = 0, -1, -2, -3, -4, -5, -6
SG_ECANCELED = -7
SG_PENDING = 1
SG_REQ_SA, SG_REQ_PT = 0, 1
SG_MEM_HOST, SG_MEM_DEVICE = 0, 1
SG_SCHEDULE_LINEAR, SG_SCHEDULE_GEOMETRIC = 0, 1
SG_JMAX = 2
SG_NOALLOC_SCRATCH_BYTES = 16 * 1024 * 1024

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()')")
_lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p


class InstanceDesc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("gauge", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("class_prob", ctypes.c_double * 3)]


class SAParams(ctypes.Structure):
    _fields_ = [("replicas", ctypes.c_int32), ("sweeps", ctypes.c_int32),
                ("beta0", ctypes.c_double), ("beta1", ctypes.c_double),
                ("schedule", ctypes.c_int32), ("instance_id", ctypes.c_uint32),
                ("seed", ctypes.c_uint64)]


class SAResult(ctypes.Structure):
    _fields_ = [("E", _P), ("eps", _P), ("spins", _P), ("spins_mem", ctypes.c_int32)]


class PTParams(ctypes.Structure):
    _fields_ = [("temps", ctypes.c_int32), ("sweeps", ctypes.c_int32),
                ("beta_min", ctypes.c_double), ("beta_max", ctypes.c_double),
                ("instance_id", ctypes.c_uint32), ("seed", ctypes.c_uint64)]


class PTResult(ctypes.Structure):
    _fields_ = [("E", _P), ("perm", _P), ("accepts", _P), ("minE", ctypes.c_int64),
                ("min_eps", ctypes.c_double), ("spins", _P), ("spins_mem", ctypes.c_int32)]


class FragmentParams(ctypes.Structure):
    _fields_ = [("l", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("beta0", ctypes.c_double),
                ("beta1", ctypes.c_double), ("instance_id", ctypes.c_uint32), ("seed", ctypes.c_uint64)]


class FragmentResult(ctypes.Structure):
    _fields_ = [("E", ctypes.c_int64), ("eps", ctypes.c_double), ("spins", _P), ("spins_mem", ctypes.c_int32)]


# the SG_KERNEL_* kinds of sg.h, in order ("sweep_chunk": many sweeps per launch)
KERNEL_KINDS = ("init", "energy", "sweep", "exchange", "other", "sweep_chunk")
_NK = len(KERNEL_KINDS)


class KernelStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * _NK), ("device_ms", ctypes.c_double * _NK),
                ("units", ctypes.c_int64 * _NK)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_active", ctypes.c_int32),
                ("chunk_sweeps", ctypes.c_int32), ("queue_capacity", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("instance", InstanceDesc), ("width", ctypes.c_int32),
                ("sweeps_per_restart", ctypes.c_int32), ("beta0", ctypes.c_double),
                ("beta1", ctypes.c_double), ("schedule", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("eps_target", ctypes.c_double), ("sweep_cap", ctypes.c_int64)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reached", ctypes.c_int32), ("sweeps", ctypes.c_int64),
                ("minE", ctypes.c_int64), ("e_gs", ctypes.c_int64), ("min_eps", ctypes.c_double),
                ("queue_s", ctypes.c_double), ("run_s", ctypes.c_double), ("total_s", ctypes.c_double)]


_SIGS = {
    "sg_instance_create": [ctypes.POINTER(InstanceDesc), ctypes.POINTER(_P)],
    "sg_instance_create_from_couplings": [ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int64,
                                          ctypes.POINTER(_P)],
    "sg_instance_get": [_P, _P, _P, _P, _P],
    "sg_instance_destroy": [_P],
    "sg_sa_run": [_P, ctypes.POINTER(SAParams), ctypes.POINTER(SAResult), _P],
    "sg_sa_run_batch": [_P, _P, ctypes.c_int32, _P, _P],
    "sg_pt_run": [_P, ctypes.POINTER(PTParams), ctypes.POINTER(PTResult), _P],
    "sg_pt_run_batch": [_P, _P, ctypes.c_int32, _P, _P],
    "sg_energy": [_P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P],
    "sg_fragment_run_batch": [_P, _P, ctypes.c_int32, _P, _P],
    "sg_fragment_tropical_run_batch": [_P, _P, ctypes.c_int32, _P, _P],
    "sg_fragment_run": [_P, ctypes.POINTER(FragmentParams), ctypes.POINTER(FragmentResult), _P],
    "sg_energy_noalloc": [ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _P],
    "sg_version": [],
    "sg_stats_enable": [ctypes.c_int32],
    "sg_stats_read": [ctypes.POINTER(KernelStats), ctypes.c_int32],
    "sg_philox_rate": [ctypes.c_int32, ctypes.POINTER(ctypes.c_double), _P],
    "sg_server_create": [ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)],
    "sg_submit": [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)],
    "sg_poll": [_P, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(Result)],
    "sg_cancel": [_P, ctypes.c_uint64],
    "sg_server_destroy": [_P],
    "sg_request_bytes": [ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)],
}
for _name, _args in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = ctypes.c_int32
_lib.sg_last_error_string.argtypes = []
_lib.sg_last_error_string.restype = ctypes.c_char_p

EXPORTED = list(_SIGS) + ["sg_last_error_string"]


class SGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libsg error {code}: {msg}")
        self.code = code


def _check(rc: int):
    if rc != SG_OK:
        raise SGError(rc, _lib.sg_last_error_string().decode())


def last_error_string() -> str:
    return _lib.sg_last_error_string().decode()


def version() -> int:
    return int(_lib.sg_version())


def _np_ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_P)


def _stream_handle(stream):
    """cudaStream_t of `stream` (a torch.cuda.Stream), else torch's current stream."""
    if stream is not None:
        return _P(stream.cuda_stream)
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return _P(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return _P(0)


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


class Instance:
    """Owned sg_instance handle (tile-planted, or wrapped couplings)."""

    def __init__(self, handle: int):
        self._h = _P(handle)
        L = ctypes.c_int32()
        egs = ctypes.c_int64()
        _check(_lib.sg_instance_get(self._h, ctypes.byref(L), None, None, ctypes.byref(egs)))
        self.L = int(L.value)
        self.N = self.L ** 3
        self.e_gs = int(egs.value)

    @classmethod
    def create(cls, L: int, seed: int, class_prob=(1 / 3, 1 / 3, 1 / 3), gauge: bool = True):
        d = InstanceDesc(L, int(bool(gauge)), seed, (ctypes.c_double * 3)(*class_prob))
        h = _P()
        _check(_lib.sg_instance_create(ctypes.byref(d), ctypes.byref(h)))
        return cls(h.value)

    @classmethod
    def from_couplings(cls, L: int, J3, e_gs: int = 0):
        """J3: int8 (L^3, 3), numpy (host) or torch CUDA tensor (device)."""
        h = _P()
        if _is_torch_cuda(J3):
            assert J3.is_contiguous() and J3.numel() == 3 * L ** 3
            _check(_lib.sg_instance_create_from_couplings(L, _P(J3.data_ptr()), SG_MEM_DEVICE,
                                                          e_gs, ctypes.byref(h)))
        else:
            J3 = np.ascontiguousarray(J3, dtype=np.int8)
            assert J3.size == 3 * L ** 3
            _check(_lib.sg_instance_create_from_couplings(L, _np_ptr(J3), SG_MEM_HOST, e_gs,
                                                          ctypes.byref(h)))
        return cls(h.value)

    def get(self):
        """-> (J3 int8 (N,3), planted int8 (N,), e_gs)."""
        J3 = np.zeros((self.N, 3), dtype=np.int8)
        planted = np.zeros(self.N, dtype=np.int8)
        egs = ctypes.c_int64()
        _check(_lib.sg_instance_get(self._h, None, _np_ptr(J3), _np_ptr(planted), ctypes.byref(egs)))
        return J3, planted, int(egs.value)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.sg_instance_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _spins_target(spins, n_rows: int, N: int):
    """spins: None | 'host' | 'device' | numpy array | torch CUDA tensor -> (obj, ptr, mem)."""
    if spins is None:
        return None, None, SG_MEM_HOST
    if isinstance(spins, str):
        if spins == "host":
            spins = np.zeros((n_rows, N), dtype=np.int8)
        elif spins == "device":
            import torch
            spins = torch.empty((n_rows, N), dtype=torch.int8, device="cuda")
        else:
            raise ValueError(spins)
    if _is_torch_cuda(spins):
        assert spins.is_contiguous() and spins.numel() == n_rows * N
        return spins, _P(spins.data_ptr()), SG_MEM_DEVICE
    assert spins.dtype == np.int8 and spins.flags["C_CONTIGUOUS"] and spins.size == n_rows * N
    return spins, _np_ptr(spins), SG_MEM_HOST


def _sa_params(replicas, sweeps, beta0, beta1, schedule, seed, instance_id):
    sch = {"linear": SG_SCHEDULE_LINEAR, "geometric": SG_SCHEDULE_GEOMETRIC}.get(schedule, schedule)
    return SAParams(replicas, sweeps, beta0, beta1, sch, instance_id, seed)


def sa_run_batch(insts, params, spins=None, stream=None):
    """Anneal several instances in one call.

    params: list of dicts with keys replicas, sweeps, beta0, beta1, schedule, seed,
    instance_id.  spins: None, 'host', 'device', or a list of per-instance targets.
    Returns a list of dicts {E, eps, spins}.
    """
    n = len(insts)
    HandleArr = _P * n
    handles = HandleArr(*[i.handle.value for i in insts])
    ps = (SAParams * n)(*[_sa_params(**p) for p in params])
    outs = (SAResult * n)()
    keep = []
    for a, (inst, p) in enumerate(zip(insts, params)):
        E = np.zeros(p["replicas"], dtype=np.int64)
        eps = np.zeros(p["replicas"], dtype=np.float64)
        tgt = spins[a] if isinstance(spins, (list, tuple)) else spins
        obj, ptr, mem = _spins_target(tgt, p["replicas"], inst.N)
        outs[a] = SAResult(_np_ptr(E), _np_ptr(eps), ptr, mem)
        keep.append({"E": E, "eps": eps, "spins": obj})
    _check(_lib.sg_sa_run_batch(handles, ps, n, outs, _stream_handle(stream)))
    return keep


def sa_run(inst: Instance, replicas: int, sweeps: int, beta0: float, beta1: float,
           schedule="linear", seed: int = 0, instance_id: int = 0, spins=None, stream=None):
    p = dict(replicas=replicas, sweeps=sweeps, beta0=beta0, beta1=beta1, schedule=schedule,
             seed=seed, instance_id=instance_id)
    return sa_run_batch([inst], [p], spins=[spins], stream=stream)[0]


def fragment_run_batch(insts, params, spins=None, stream=None, tropical=False):
    """The fragment meta-heuristic (Sec. II; App. A) with SA fragment anneals, on
    instances of one side L.  params: list of dicts with keys l, sweeps, beta0, beta1,
    seed, instance_id (l, sweeps and betas equal across the batch).  spins: None,
    'host', 'device' or a list of per-instance targets.  tropical: the centre spins set
    by exact zero-temperature cube marginals instead (l in {1, 3}; sweeps and betas
    unused).  Returns a list of dicts {E, eps, spins}."""
    n = len(insts)
    handles = (_P * n)(*[i.handle.value for i in insts])
    ps = (FragmentParams * n)(*[FragmentParams(p["l"], p.get("sweeps", 0), p.get("beta0", 1.0), p.get("beta1", 1.0),
                                               p.get("instance_id", 0), p.get("seed", 0)) for p in params])
    outs = (FragmentResult * n)()
    keep = []
    for a, inst in enumerate(insts):
        tgt = spins[a] if isinstance(spins, (list, tuple)) else spins
        obj, ptr, mem = _spins_target(tgt, 1, inst.N)
        outs[a] = FragmentResult(0, 0.0, ptr, mem)
        keep.append(obj)
    fn = _lib.sg_fragment_tropical_run_batch if tropical else _lib.sg_fragment_run_batch
    _check(fn(handles, ps, n, outs, _stream_handle(stream)))
    res = []
    for a in range(n):
        sp = keep[a]
        if sp is not None:
            sp = sp.reshape(-1)
        res.append({"E": int(outs[a].E), "eps": float(outs[a].eps), "spins": sp})
    return res


def fragment_run(inst: Instance, l: int, sweeps: int, beta0: float, beta1: float, seed: int = 0,
                 instance_id: int = 0, spins=None, stream=None):
    p = dict(l=l, sweeps=sweeps, beta0=beta0, beta1=beta1, seed=seed, instance_id=instance_id)
    return fragment_run_batch([inst], [p], spins=[spins], stream=stream)[0]


def fragment_tropical_run(inst: Instance, l: int, spins=None, stream=None):
    return fragment_run_batch([inst], [dict(l=l)], spins=[spins], stream=stream, tropical=True)[0]


def pt_run_batch(insts, params, spins=None, stream=None):
    """Parallel tempering of several instances.  params: dicts with temps, sweeps,
    beta_min, beta_max, seed, instance_id.  Returns dicts {E, perm, accepts, minE,
    min_eps, spins} (E, perm, spins by slot)."""
    n = len(insts)
    handles = (_P * n)(*[i.handle.value for i in insts])
    ps = (PTParams * n)(*[PTParams(p["temps"], p["sweeps"], p["beta_min"], p["beta_max"],
                                   p.get("instance_id", 0), p.get("seed", 0)) for p in params])
    outs = (PTResult * n)()
    keep = []
    for a, (inst, p) in enumerate(zip(insts, params)):
        K = p["temps"]
        E = np.zeros(K, dtype=np.int64)
        perm = np.zeros(K, dtype=np.int32)
        acc = np.zeros(max(K - 1, 1), dtype=np.int64)
        tgt = spins[a] if isinstance(spins, (list, tuple)) else spins
        obj, ptr, mem = _spins_target(tgt, K, inst.N)
        outs[a] = PTResult(_np_ptr(E), _np_ptr(perm), _np_ptr(acc), 0, 0.0, ptr, mem)
        keep.append({"E": E, "perm": perm, "accepts": acc[: max(K - 1, 0)], "spins": obj})
    _check(_lib.sg_pt_run_batch(handles, ps, n, outs, _stream_handle(stream)))
    for a in range(n):
        keep[a]["minE"] = int(outs[a].minE)
        keep[a]["min_eps"] = float(outs[a].min_eps)
    return keep


def pt_run(inst: Instance, temps: int, sweeps: int, beta_min: float, beta_max: float,
           seed: int = 0, instance_id: int = 0, spins=None, stream=None):
    p = dict(temps=temps, sweeps=sweeps, beta_min=beta_min, beta_max=beta_max, seed=seed,
             instance_id=instance_id)
    return pt_run_batch([inst], [p], spins=[spins], stream=stream)[0]


def energy(inst: Instance, spins, stream=None) -> np.ndarray:
    """Energies (Eq. 1) of configurations spins (n, N): numpy host or torch CUDA."""
    if _is_torch_cuda(spins):
        assert spins.is_contiguous() and spins.numel() % inst.N == 0
        n = spins.numel() // inst.N
        ptr, mem = _P(spins.data_ptr()), SG_MEM_DEVICE
    else:
        spins = np.ascontiguousarray(spins, dtype=np.int8)
        n = spins.size // inst.N
        ptr, mem = _np_ptr(spins), SG_MEM_HOST
    E = np.zeros(n, dtype=np.int64)
    _check(_lib.sg_energy(inst.handle, ptr, n, mem, _np_ptr(E), _stream_handle(stream)))
    return E


def stats_enable(timing: bool):
    """Time every later launch with CUDA events on its own stream (process-wide)."""
    _check(_lib.sg_stats_enable(int(bool(timing))))


def stats_read(reset: bool = False) -> dict:
    """Launch counts, summed device milliseconds and work units per kernel kind."""
    st = KernelStats()
    _check(_lib.sg_stats_read(ctypes.byref(st), int(bool(reset))))
    return {k: {"launches": int(st.launches[i]), "device_ms": float(st.device_ms[i]),
                "units": int(st.units[i])} for i, k in enumerate(KERNEL_KINDS)}


def philox_rate(blocks_per_thread: int = 4096, stream=None) -> float:
    """Philox4x32-10 blocks per second this device produces when drawing is all it does
    (16 x this bounds the sweeps' attempt rate: two blocks per word of 32 replicas)."""
    out = ctypes.c_double()
    _check(_lib.sg_philox_rate(int(blocks_per_thread), ctypes.byref(out), _stream_handle(stream)))
    return out.value


def _check_noalloc_args(L: int, J3_dev, spins_dev, E_dev) -> int:
    """Validates the tensors of energy_noalloc before anything reaches the device; returns
    the number of configurations.  Raises ValueError (not an assert, so it holds under -O)."""
    import torch
    if not isinstance(L, int) or L < 2 or L % 2 or L > 256:
        raise ValueError(f"L must be an even int in [2, 256], got {L!r}")
    N = L ** 3
    named = (("J3_dev", J3_dev, torch.int8), ("spins_dev", spins_dev, torch.int8), ("E_dev", E_dev, torch.int64))
    for name, t, dt in named:
        if not _is_torch_cuda(t):
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must have dtype {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    dev = torch.cuda.current_device()
    for name, t, _ in named:
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
    if J3_dev.numel() != 3 * N:
        raise ValueError(f"J3_dev must hold L^3 x 3 = {3 * N} couplings, got {J3_dev.numel()}")
    n = spins_dev.numel() // N
    if n < 1 or spins_dev.numel() != n * N:
        raise ValueError(f"spins_dev must hold a positive multiple of L^3 = {N} spins, got {spins_dev.numel()}")
    if E_dev.numel() != n:
        raise ValueError(f"E_dev must hold one energy per configuration ({n}), got {E_dev.numel()}")
    return n


def energy_noalloc(L: int, J3_dev, spins_dev, E_dev, stream=None):
    """Energies of spins_dev (n, L^3) into E_dev (n,) int64, all torch CUDA tensors on the
    current device, through the entry point that allocates no device memory (for callers
    that cannot let a library allocate: it uses a fixed scratch array instead)."""
    n = _check_noalloc_args(L, J3_dev, spins_dev, E_dev)
    _check(_lib.sg_energy_noalloc(L, _P(J3_dev.data_ptr()), _P(spins_dev.data_ptr()), n,
                                  _P(E_dev.data_ptr()), _stream_handle(stream)))


def request(kind: int, L: int, seed: int, width: int, beta0: float, beta1: float, eps_target: float,
            sweep_cap: int, run_seed: int = 0, sweeps_per_restart: int = 1000,
            schedule: int = SG_SCHEDULE_LINEAR, class_prob=(1 / 3, 1 / 3, 1 / 3),
            gauge: bool = True) -> Request:
    """A solve request: a fresh tile-planted instance (L, seed, class_prob, gauge) solved by
    SA (width replicas, restarts of sweeps_per_restart sweeps) or PT (width temperatures)
    until its gap reaches eps_target (Eq. 2) or sweep_cap sweeps have run."""
    d = InstanceDesc(L, int(bool(gauge)), seed, (ctypes.c_double * 3)(*class_prob))
    return Request(kind, d, width, sweeps_per_restart, beta0, beta1, schedule, run_seed, eps_target,
                   sweep_cap)


def request_bytes(req: Request) -> int:
    """Device memory a server holds for `req` while it runs (what admission counts)."""
    b = ctypes.c_uint64()
    _check(_lib.sg_request_bytes(ctypes.byref(req), ctypes.byref(b)))
    return int(b.value)


class Server:
    """Continuously batched solve server on the current CUDA device (sg_server_*)."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 64, chunk_sweeps: int = 50,
                 queue_capacity: int = 1 << 16):
        self._h = _P()
        cfg = ServerConfig(hbm_budget_bytes, max_active, chunk_sweeps, queue_capacity)
        _check(_lib.sg_server_create(ctypes.byref(cfg), ctypes.byref(self._h)))

    def submit(self, req: Request) -> int:
        t = ctypes.c_uint64()
        _check(_lib.sg_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int, timeout_ms: int = -1):
        """The result as a dict once done (reported once), else None."""
        r = Result()
        rc = _lib.sg_poll(self._h, ticket, timeout_ms, ctypes.byref(r))
        if rc == SG_PENDING:
            return None
        _check(rc)
        return {f: getattr(r, f) for f, _ in Result._fields_}

    def cancel(self, ticket: int):
        _check(_lib.sg_cancel(self._h, ticket))

    def close(self):
        if self._h:
            _check(_lib.sg_server_destroy(self._h))
            self._h = _P()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
