"""Python binding of the tnmc C ABI (``include/tnmc.h``): argument marshalling only.

Every step of the slice update runs in the CUDA library ``_lib/libtnmc.so``;
this module converts arrays and torch tensors to pointers and raises on error
codes. There is no CPU fallback: without the built library or a CUDA device
every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

from . import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libtnmc.so")

PREC_F64, PREC_F32, PREC_BF16 = 0, 1, 2
FIX_R1, FIX_R2 = 0, 1
PROPOSAL_TN, PROPOSAL_NET, PROPOSAL_CACHE = 0, 1, 2
ROUTE_LQ, ROUTE_DM = 0, 1

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_ADJACENT", 3: "ERR_OOM", 4: "ERR_CUDA", 5: "ERR_TIMEOUT",
          6: "ERR_NONFINITE", 7: "ERR_STATE"}


class TnmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tnmc {STATUS.get(code, code)}: {msg}")
        self.code = code


class Tuning(C.Structure):
    """Kernel configuration of a context (see tnmc_tuning in include/tnmc.h); -1 keeps a field."""
    _fields_ = [("gemm_mode", C.c_int), ("eig_smem", C.c_int), ("jac_floor", C.c_int), ("ctas_per_sm", C.c_int),
                ("route", C.c_int), ("gemm_tile", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class _Config(C.Structure):
    _fields_ = [("Lx", C.c_int), ("Ly", C.c_int), ("Lz", C.c_int), ("bc", C.c_int * 3), ("model", C.c_int),
                ("q", C.c_int), ("chi", C.c_int), ("precision", C.c_int), ("fix_mode", C.c_int),
                ("n_chains", C.c_int), ("betas", C.POINTER(C.c_double)),
                ("instance_of_chain", C.POINTER(C.c_int32)), ("n_inst", C.c_int),
                ("couplings", C.POINTER(C.c_int32)), ("couplings_on_device", C.c_int), ("layers", C.c_int)]


_lib = None

# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("tnmc_create", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(_Config), C.c_int, C.c_void_p]),
    ("tnmc_set_spins", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    ("tnmc_get_spins", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    ("tnmc_slice_update", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int32),
                                    C.POINTER(C.c_int32), C.c_uint64, C.c_uint64, C.c_int, C.c_int,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("tnmc_sweep", C.c_int, [C.c_void_p, C.c_int, C.c_uint64, C.c_int, C.c_void_p]),
    ("tnmc_get_sweep", C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    ("tnmc_set_sweep", C.c_int, [C.c_void_p, C.c_uint64]),
    ("tnmc_observables", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int32), C.c_void_p]),
    ("tnmc_slice_logz", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint64,
                                  C.POINTER(C.c_double)]),
    ("tnmc_set_proposal_beta_factor", C.c_int, [C.c_void_p, C.c_double]),
    ("tnmc_sync", C.c_int, [C.c_void_p]),
    ("tnmc_set_proposals_per_env", C.c_int, [C.c_void_p, C.c_int]),
    ("tnmc_cache_build", C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64]),
    ("tnmc_set_cache_mix", C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    ("tnmc_metropolis_sweep", C.c_int, [C.c_void_p, C.c_int, C.c_uint64, C.c_void_p]),
    ("tnmc_events", C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    ("tnmc_memory", C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    ("tnmc_save", C.c_int, [C.c_void_p, C.c_char_p]),
    ("tnmc_load", C.c_int, [C.c_void_p, C.c_char_p]),
    ("tnmc_net_init", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_uint64, C.c_int]),
    ("tnmc_net_param_count", C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    ("tnmc_net_set_params", C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    ("tnmc_net_get_params", C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    ("tnmc_set_proposal_mix", C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    ("tnmc_net_buffer_count", C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    ("tnmc_net_train", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_float, C.c_uint64, C.POINTER(C.c_double)]),
    ("tnmc_net_adam_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_float]),
    ("tnmc_net_eval", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                C.c_uint64, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("tnmc_slice_logz_noalloc", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                          C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint64,
                                          C.c_int, C.c_void_p, C.c_void_p]),
    ("tnmc_set_tuning", C.c_int, [C.c_void_p, C.c_void_p]),
    ("tnmc_get_tuning", C.c_int, [C.c_void_p, C.c_void_p]),
    ("tnmc_probe_alu_peak", C.c_int, [C.c_int, C.c_void_p, C.POINTER(C.c_double)]),
    ("tnmc_cta_gemm", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, C.c_void_p, C.c_int,
                                C.c_longlong, C.c_int, C.c_void_p, C.c_int, C.c_longlong, C.c_int, C.c_float,
                                C.c_void_p, C.c_int, C.c_longlong, C.c_void_p]),
    ("tnmc_last_error", C.c_char_p, [C.c_void_p]),
    ("tnmc_destroy", None, [C.c_void_p]),
]


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"tnmc CUDA library not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _items(chains, slices):
    """(chain, slice) item arrays as int32, checked to be 1-D and of equal length (the C ABI reads
    n_items entries of each)."""
    chains = np.ascontiguousarray(chains, dtype=np.int32)
    slices = np.ascontiguousarray(slices, dtype=np.int32)
    if chains.ndim != 1 or chains.shape != slices.shape:
        raise ValueError(f"chains and slices must be 1-D of equal length, got {chains.shape} and {slices.shape}")
    return chains, slices


def _expect_shape(name, shape, expected):
    if tuple(shape) != tuple(expected):
        raise ValueError(f"{name}: expected shape {tuple(expected)}, got {tuple(shape)}")


def _check_counter(counter, n_chains):
    """The sweep kernels add one count per accepted slice at counter[global chain] on the device."""
    if counter is None:
        return
    if not (getattr(counter, "is_cuda", False) and str(counter.dtype) == "torch.int32" and counter.is_contiguous()):
        raise ValueError("accept_counter must be a contiguous int32 CUDA tensor")
    if counter.numel() < n_chains:
        raise ValueError(f"accept_counter has {counter.numel()} entries, the context has {n_chains} chains")


class Context:
    """A tnmc context over one or more workloads (lattice groups) on the current CUDA device.

    layers = 2 makes every group update TNMCMC-2 composite layers of superspins (Ising only)."""

    def __init__(self, workloads: Sequence[inputs.Workload], precision: int = PREC_F64, fix_mode: int = FIX_R1,
                 stream=None, layers: int = 1):
        import torch

        self.lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("tnmc needs a CUDA device")
        self.torch = torch
        self.workloads = list(workloads)
        cfgs = (_Config * len(self.workloads))()
        self._keep = []
        for i, wl in enumerate(self.workloads):
            betas = np.ascontiguousarray(wl.chain_beta(), dtype=np.float64)
            inst = np.ascontiguousarray(wl.chain_instance(), dtype=np.int32)
            J = np.ascontiguousarray(wl.couplings, dtype=np.int32)
            self._keep += [betas, inst, J]
            c = cfgs[i]
            c.Lx, c.Ly, c.Lz = wl.dims
            for a in range(3):
                c.bc[a] = int(wl.bc[a])
            c.model = wl.model
            c.q = wl.potts_q
            c.chi = wl.chi
            c.precision = precision
            c.fix_mode = fix_mode
            c.n_chains = wl.n_chains
            c.betas = betas.ctypes.data_as(C.POINTER(C.c_double))
            c.instance_of_chain = inst.ctypes.data_as(C.POINTER(C.c_int32))
            c.n_inst = wl.n_inst
            c.couplings = J.ctypes.data_as(C.POINTER(C.c_int32))
            c.couplings_on_device = 0
            c.layers = layers
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        st = self.lib.tnmc_create(C.byref(h), cfgs, len(self.workloads), C.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise TnmcError(st, "tnmc_create failed")
        self.h = h
        self._keep = []
        self.precision = precision
        self.layers = layers
        self.lmax = max(max(wl.dims) for wl in self.workloads)

    # ------------------------------------------------------------------ utils
    def _check(self, st):
        if st != 0:
            raise TnmcError(st, self.lib.tnmc_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.tnmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ state
    def set_spins(self, group: int, spins):
        t = self.torch
        wl = self.workloads[group]
        _expect_shape("spins", spins.shape, (wl.n_chains, wl.dims[2], wl.dims[1], wl.dims[0]))
        if isinstance(spins, np.ndarray):
            arr = np.ascontiguousarray(spins, dtype=np.int8)
            self._check(self.lib.tnmc_set_spins(self.h, group, arr.ctypes.data_as(C.c_void_p), 0))
        else:
            ts = spins.to(dtype=t.int8).contiguous()
            self._check(self.lib.tnmc_set_spins(self.h, group, _ptr(ts), 1 if ts.is_cuda else 0))

    def get_spins(self, group: int) -> np.ndarray:
        wl = self.workloads[group]
        out = np.zeros((wl.n_chains, wl.dims[2], wl.dims[1], wl.dims[0]), dtype=np.int8)
        self._check(self.lib.tnmc_get_spins(self.h, group, out.ctypes.data_as(C.c_void_p), 0))
        return out

    def get_spins_device(self, group: int):
        wl = self.workloads[group]
        out = self.torch.empty((wl.n_chains, wl.dims[2], wl.dims[1], wl.dims[0]), dtype=self.torch.int8,
                               device="cuda")
        self._check(self.lib.tnmc_get_spins(self.h, group, _ptr(out), 1))
        return out

    # ------------------------------------------------------------ the hot path
    def slice_update(self, group: int, axis: int, chains, slices, seed: int, step: int, write_back: bool = True,
                     proposal: int = PROPOSAL_TN, want_spins: bool = True):
        t = self.torch
        chains, slices = _items(chains, slices)
        n = len(chains)
        dev = "cuda"
        out = {
            "logq_new": t.empty(n, dtype=t.float64, device=dev),
            "logq_old": t.empty(n, dtype=t.float64, device=dev),
            "accept": t.empty(n, dtype=t.uint8, device=dev),
            "dE": t.empty(n, dtype=t.int64, device=dev),
        }
        if want_spins:
            out["new_spins"] = t.empty((n, self.lmax, self.lmax), dtype=t.int8, device=dev)
        self._check(self.lib.tnmc_slice_update(
            self.h, group, axis, n, chains.ctypes.data_as(C.POINTER(C.c_int32)),
            slices.ctypes.data_as(C.POINTER(C.c_int32)), C.c_uint64(seed), C.c_uint64(step), proposal,
            1 if write_back else 0, _ptr(out.get("new_spins")), _ptr(out["logq_new"]), _ptr(out["logq_old"]),
            _ptr(out["accept"]), _ptr(out["dE"])))
        return out

    def sweep(self, n_sweeps: int, seed: int, use_graph: bool = False, accept_counter=None):
        _check_counter(accept_counter, sum(wl.n_chains for wl in self.workloads))
        self._check(self.lib.tnmc_sweep(self.h, n_sweeps, C.c_uint64(seed), 1 if use_graph else 0,
                                        _ptr(accept_counter)))

    @property
    def sweep_counter(self) -> int:
        v = C.c_uint64()
        self._check(self.lib.tnmc_get_sweep(self.h, C.byref(v)))
        return v.value

    @sweep_counter.setter
    def sweep_counter(self, t: int):
        self._check(self.lib.tnmc_set_sweep(self.h, C.c_uint64(t)))

    def observables(self, group: int, partner: Optional[np.ndarray] = None, out=None):
        """E/N, M and the overlap with the partner chain, [n_chains, 3] float64 on the device, written on the
        context's stream (call sync() before reading on another stream)."""
        wl = self.workloads[group]
        if out is None:
            out = self.torch.empty((wl.n_chains, 3), dtype=self.torch.float64, device="cuda")
        assert out.is_contiguous() and tuple(out.shape) == (wl.n_chains, 3)
        p = None
        if partner is not None:
            arr = np.ascontiguousarray(partner, dtype=np.int32)
            _expect_shape("partner", arr.shape, (wl.n_chains,))
            p = arr.ctypes.data_as(C.POINTER(C.c_int32))
        self._check(self.lib.tnmc_observables(self.h, group, p, _ptr(out)))
        return out

    def slice_logz(self, group: int, chain: int, axis: int, slice_: int, seed: int, step: int) -> float:
        v = C.c_double()
        self._check(self.lib.tnmc_slice_logz(self.h, group, chain, axis, slice_, C.c_uint64(seed),
                                             C.c_uint64(step), C.byref(v)))
        return v.value

    def get_tuning(self) -> dict:
        t = Tuning()
        self._check(self.lib.tnmc_get_tuning(self.h, C.byref(t)))
        return t.as_dict()

    def set_tuning(self, gemm_mode=-1, eig_smem=-1, jac_floor=-1, ctas_per_sm=-1, route=-1, gemm_tile=-1):
        t = Tuning(gemm_mode, eig_smem, jac_floor, ctas_per_sm, route, gemm_tile)
        self._check(self.lib.tnmc_set_tuning(self.h, C.byref(t)))

    def set_proposal_beta_factor(self, f: float):
        self._check(self.lib.tnmc_set_proposal_beta_factor(self.h, C.c_double(f)))

    def sync(self):
        self._check(self.lib.tnmc_sync(self.h))

    def metropolis_sweep(self, n_sweeps: int, seed: int, accept_counter=None):
        """Single-spin checkerboard Metropolis sweeps of every chain (the paper's comparison method)."""
        _check_counter(accept_counter, sum(wl.n_chains for wl in self.workloads))
        self._check(self.lib.tnmc_metropolis_sweep(self.h, n_sweeps, C.c_uint64(seed), _ptr(accept_counter)))

    def set_proposals_per_env(self, n_prop: int):
        """Tensor-network proposals per environment build (1 = Algorithm 2)."""
        self._check(self.lib.tnmc_set_proposals_per_env(self.h, n_prop))

    def cache_build(self, seed: int, step: int):
        """Contract and keep the environments of every chain, axis and slice for the current spins (fixed
        lines drawn for (seed, step)); slice_update(proposal=PROPOSAL_CACHE) and sweeps after
        set_cache_mix(True, k) propose from them."""
        self._check(self.lib.tnmc_cache_build(self.h, C.c_uint64(seed), C.c_uint64(step)))

    def set_cache_mix(self, on: bool, fresh_every: int = 0):
        """Sweeps propose from the cache (on), contracting afresh on sweeps t with t % k == k - 1 for
        k = fresh_every > 0."""
        self._check(self.lib.tnmc_set_cache_mix(self.h, 1 if on else 0, fresh_every))

    def events(self) -> int:
        """Sites whose conditional fell back to the uniform distribution so far."""
        v = C.c_uint64()
        self._check(self.lib.tnmc_events(self.h, C.byref(v)))
        return v.value

    def memory_bytes(self) -> int:
        v = C.c_size_t()
        self._check(self.lib.tnmc_memory(self.h, C.byref(v)))
        return v.value

    # ------------------------------------------------------- learned proposal
    def net_init(self, channels: int = 64, layers: int = 6, seed: int = 0, buffer_slots: int = 4096):
        self._check(self.lib.tnmc_net_init(self.h, channels, layers, C.c_uint64(seed), buffer_slots))

    def net_param_count(self) -> int:
        v = C.c_size_t()
        self._check(self.lib.tnmc_net_param_count(self.h, C.byref(v)))
        return v.value

    def net_set_params(self, w: np.ndarray):
        arr = np.ascontiguousarray(w, dtype=np.float32)
        assert arr.size == self.net_param_count()
        self._check(self.lib.tnmc_net_set_params(self.h, arr.ctypes.data_as(C.c_void_p), 0))

    def net_get_params(self) -> np.ndarray:
        out = np.zeros(self.net_param_count(), dtype=np.float32)
        self._check(self.lib.tnmc_net_get_params(self.h, out.ctypes.data_as(C.c_void_p), 0))
        return out

    def set_proposal_mix(self, net_every: int, record: bool):
        self._check(self.lib.tnmc_set_proposal_mix(self.h, net_every, 1 if record else 0))

    def net_buffer_count(self) -> int:
        v = C.c_uint64()
        self._check(self.lib.tnmc_net_buffer_count(self.h, C.byref(v)))
        return v.value

    def net_train(self, n_steps: int, batch: int, lr: float, seed: int) -> np.ndarray:
        losses = np.zeros(n_steps, dtype=np.float64)
        self._check(self.lib.tnmc_net_train(self.h, n_steps, batch, C.c_float(lr), C.c_uint64(seed),
                                            losses.ctypes.data_as(C.POINTER(C.c_double))))
        return losses

    def net_adam_step(self, grad: np.ndarray, lr: float):
        """One Adam step of the network's parameters with a given gradient (host array [n_params])."""
        arr = np.ascontiguousarray(grad, dtype=np.float32)
        _expect_shape("grad", arr.shape, (self.net_param_count(),))
        self._check(self.lib.tnmc_net_adam_step(self.h, arr.ctypes.data_as(C.c_void_p), 0, C.c_float(lr)))

    def net_eval(self, group, axis, chains, slices, seed, step, logits=True, grad=False):
        """Teacher-forced network pass on the current slices: logits [n, d, Lmax^2] (compact raster
        positions r * Lc + x first), log q [n], and optionally the gradient of the mean NLL."""
        t = self.torch
        chains, slices = _items(chains, slices)
        n = len(chains)
        d = self.workloads[group].d
        out = {"logq": t.empty(n, dtype=t.float64, device="cuda")}
        if logits:
            out["logits"] = t.empty((n, d, self.lmax * self.lmax), dtype=t.float32, device="cuda")
        if grad:
            out["grad"] = t.empty(self.net_param_count(), dtype=t.float32, device="cuda")
        self._check(self.lib.tnmc_net_eval(self.h, group, axis, n, chains.ctypes.data_as(C.POINTER(C.c_int32)),
                                           slices.ctypes.data_as(C.POINTER(C.c_int32)), C.c_uint64(seed),
                                           C.c_uint64(step), _ptr(out.get("logits")), _ptr(out["logq"]),
                                           _ptr(out.get("grad"))))
        return out

    def save(self, path: str):
        self._check(self.lib.tnmc_save(self.h, path.encode()))

    def load(self, path: str):
        self._check(self.lib.tnmc_load(self.h, path.encode()))


def _check_device_tensor(name, t, dtype, shape=None, min_numel=None):
    """A tensor handed to the C ABI as a raw device pointer: on the current CUDA device, contiguous, of the
    expected dtype and shape (the kernel reads or writes exactly that many elements)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{torch.cuda.current_device()}")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None:
        _expect_shape(name, t.shape, shape)
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError(f"{name} needs at least {min_numel} elements, got {t.numel()}")


def slice_logz_noalloc(spins, couplings, dims, bc, model: int, beta: float, chi: int, axis: int, slice_: int,
                       seed: int, step: int, fix_mode: int = FIX_R1, out=None, stream=None):
    """log Z of one slice without a context or any allocation inside the library.

    spins: CUDA int8 tensor [Lz, Ly, Lx]; couplings: CUDA int32 tensor [3, Lz, Ly, Lx]; out: CUDA float64
    tensor with at least one element (allocated here if None). All on the current device. Returns out; the
    caller synchronises."""
    import torch
    lib = load_library()
    Lx, Ly, Lz = (int(v) for v in dims)
    _check_device_tensor("spins", spins, torch.int8, (Lz, Ly, Lx))
    _check_device_tensor("couplings", couplings, torch.int32, (3, Lz, Ly, Lx))
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=spins.device)
    _check_device_tensor("out", out, torch.float64, min_numel=1)
    if len(bc) != 3:
        raise ValueError("bc must have 3 entries")
    bcs = (C.c_int * 3)(*[int(b) for b in bc])
    st = stream if stream is not None else torch.cuda.current_stream()
    code = lib.tnmc_slice_logz_noalloc(_ptr(spins), _ptr(couplings), Lx, Ly, Lz, bcs, model,
                                       C.c_double(beta), chi, axis, slice_, C.c_uint64(seed), C.c_uint64(step),
                                       fix_mode, _ptr(out), C.c_void_p(st.cuda_stream))
    if code != 0:
        raise TnmcError(code, "tnmc_slice_logz_noalloc")
    return out


def probe_alu_peak(precision: int, stream=None) -> float:
    """Measured FMA throughput (flop/s) of the current device's CUDA cores in FP32 or FP64."""
    import torch
    lib = load_library()
    st = stream if stream is not None else torch.cuda.current_stream()
    v = C.c_double()
    code = lib.tnmc_probe_alu_peak(precision, C.c_void_p(st.cuda_stream), C.byref(v))
    if code != 0:
        raise TnmcError(code, "tnmc_probe_alu_peak")
    return v.value


GEMM_FFMA, GEMM_MMA_TF32X3, GEMM_MMA_BF16, GEMM_UMMA_TF32X3, GEMM_UMMA_BF16 = 0, 1, 2, 3, 4


def cta_gemm(engine: int, a, b, c, alpha: float = 1.0, beta: float = 0.0, trans_a: bool = False,
             trans_b: bool = False, stream=None):
    """C[i] = alpha op(A[i]) op(B[i]) + beta C[i] with one CTA per matrix, on the selected GEMM engine.

    a, b, c: contiguous CUDA float32 tensors [batch, rows, cols] (op(A) = A^T when trans_a, and so on).
    Returns c (written in place); the call synchronises the stream."""
    import torch
    lib = load_library()
    for name, t in (("a", a), ("b", b), ("c", c)):
        _check_device_tensor(name, t, torch.float32)
        if t.dim() != 3:
            raise ValueError(f"{name} must be [batch, rows, cols]")
    batch = c.shape[0]
    if a.shape[0] != batch or b.shape[0] != batch:
        raise ValueError("a, b and c need the same batch size")
    M, N = c.shape[1], c.shape[2]
    K = a.shape[1] if trans_a else a.shape[2]
    if (a.shape[2] if trans_a else a.shape[1]) != M or (b.shape[2] if trans_b else b.shape[1]) != K or \
            (b.shape[1] if trans_b else b.shape[2]) != N:
        raise ValueError("shapes of a, b and c do not match")
    st = stream if stream is not None else torch.cuda.current_stream()
    code = lib.tnmc_cta_gemm(engine, batch, M, N, K, C.c_float(alpha), _ptr(a), max(1, a.shape[2]),
                             a.shape[1] * a.shape[2], int(trans_a), _ptr(b), max(1, b.shape[2]),
                             b.shape[1] * b.shape[2], int(trans_b), C.c_float(beta), _ptr(c), max(1, N), M * N,
                             C.c_void_p(st.cuda_stream))
    if code != 0:
        raise TnmcError(code, "tnmc_cta_gemm")
    return c


def colour_classes(n: int, periodic: bool) -> List[List[int]]:
    """Slices of one axis in non-adjacent groups (host-side scheduling helper)."""
    if periodic and n % 2 == 1 and n > 1:
        return [list(range(0, n - 1, 2)), list(range(1, n - 1, 2)), [n - 1]]
    return [list(range(0, n, 2)), list(range(1, n, 2))]


def composite_classes(n: int, periodic: bool, offset: int) -> List[List[int]]:
    """First layers of the TNMCMC-2 composites of one axis and offset (sweep t: offset (t // 3) % 2),
    grouped into the colour classes that tnmc_sweep runs (host-side scheduling helper)."""
    nc, ring = (n // 2, n % 2 == 0) if periodic else ((n - offset) // 2, False)
    if nc <= 0:
        return []
    return [[(offset + 2 * j) % n for j in cls] for cls in colour_classes(nc, ring)]
