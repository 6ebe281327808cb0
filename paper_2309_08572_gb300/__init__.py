"""Python binding of libmpdo (GB300 noisy neutral-atom MPDO simulator).

Argument marshalling only: every step of the method runs in the CUDA library behind the
C ABI declared in include/mpdo.h.  The library is loaded from this package directory
(built in-tree by build.py); importing this module raises if it is missing, so no code
path can fall back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmpdo.so")

MPDO_FP64, MPDO_C64, MPDO_TF32X3, MPDO_BF16X3 = 0, 1, 2, 3
PREC = {"fp64": MPDO_FP64, "c64": MPDO_C64, "tf32x3": MPDO_TF32X3, "bf16x3": MPDO_BF16X3}
ERRORS = {-1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_NUMERIC", -5: "ERR_TIMEOUT",
          -6: "ERR_STATE"}


class MpdoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [("n_sites", C.c_int), ("d", C.c_int), ("chi_max", C.c_int), ("k_max", C.c_int),
                ("m_max", C.c_int), ("prec", C.c_int), ("sv_cutoff", C.c_double),
                ("kraus_cutoff", C.c_double), ("use_ppt", C.c_int), ("cuda_stream", C.c_void_p),
                ("gram_fp64", C.c_int), ("order", C.c_int),
                ("alloc", C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)),
                ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)), ("alloc_ctx", C.c_void_p)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
ORDER = {"ltr": 0, "snake": 1}


class Op(C.Structure):
    _fields_ = [("kind", C.c_int), ("site", C.c_int), ("n_kraus", C.c_int),
                ("ops", C.POINTER(C.c_double))]


class Layer(C.Structure):
    _fields_ = [("n_ops", C.c_int), ("ops", C.POINTER(Op))]


class CircuitDesc(C.Structure):
    _fields_ = [("n_sites", C.c_int), ("chi_max", C.c_int), ("k_max", C.c_int),
                ("use_ppt", C.c_int), ("n_layers", C.c_int), ("layers", C.POINTER(C.c_void_p)),
                ("J", C.c_double), ("hx", C.c_double), ("b", C.c_double)]


class Pulse(C.Structure):
    """Gaussian pulse of the G1 CZ: times in us, angular frequencies in rad/us."""
    _fields_ = [("T", C.c_double), ("omega_max", C.c_double), ("delta", C.c_double),
                ("blockade", C.c_double), ("width", C.c_double)]


# Fig. 1 (d, e): T = 2.165 us, Omega_max = 17 MHz, Delta = -14.7 MHz, B = 60 MHz (x 2 pi)
GAUSSIAN_CZ = dict(T=2.165, omega_max=2 * np.pi * 17.0, delta=2 * np.pi * -14.7,
                   blockade=2 * np.pi * 60.0, width=0.1)


class CircuitHostDesc(C.Structure):
    _fields_ = [("n_sites", C.c_int), ("chi_max", C.c_int), ("k_max", C.c_int),
                ("use_ppt", C.c_int), ("n_layers", C.c_int), ("layers", C.POINTER(Layer)),
                ("J", C.c_double), ("hx", C.c_double), ("b", C.c_double)]


class TruncStats(C.Structure):
    _fields_ = [("disc_bond_w", C.c_double), ("disc_kraus_w", C.c_double),
                ("ppt_theta_min", C.c_double), ("ppt_infeasible", C.c_int),
                ("ppt_clamped", C.c_int), ("chi_used_max", C.c_int), ("k_used_max", C.c_int),
                ("n_updates", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(LIB_PATH)
    P, I, D, VP, S = C.POINTER, C.c_int, C.c_double, C.c_void_p, C.c_size_t
    sig = {
        "mpdo_create": (I, [P(Config), P(D), P(VP)]),
        "mpdo_reset": (I, [VP, P(D)]),
        "mpdo_apply_layer": (I, [VP, P(Layer), P(TruncStats)]),
        "mpdo_layer_upload": (I, [VP, P(Layer), P(VP)]),
        "mpdo_apply_dlayer": (I, [VP, VP, P(TruncStats)]),
        "mpdo_layer_free": (I, [VP, VP]),
        "mpdo_truncate": (I, [VP, I, I, I, P(TruncStats)]),
        "mpdo_expect_energy": (I, [VP, D, D, D, P(D), P(D), P(D), P(D)]),
        "mpdo_sample_probs": (I, [VP, I, C.c_uint64, P(C.c_uint8), P(D)]),
        "mpdo_get_dims": (I, [VP, P(I), P(I), P(I)]),
        "mpdo_vmpo_create": (I, [I, I, I, D, P(D), VP, P(VP)]),
        "mpdo_vmpo_apply_layer": (I, [VP, P(Layer), P(TruncStats)]),
        "mpdo_vmpo_expect_energy": (I, [VP, D, D, D, P(D), P(D), P(D), P(D)]),
        "mpdo_vmpo_purity": (I, [VP, P(D)]),
        "mpdo_vmpo_collision": (I, [VP, P(D)]),
        "mpdo_vmpo_set_precision": (I, [VP, I]),
        "mpdo_vmpo_get_dims": (I, [VP, P(I), P(I)]),
        "mpdo_vmpo_destroy": (I, [VP]),
        "mpdo_expect_second_order": (I, [VP, I, P(D), P(D), P(D), P(D), P(D)]),
        "mpdo_reconfigure": (I, [VP, I, I, I, I, P(D)]),
        "mpdo_batch_run": (I, [I, P(VP), I, P(CircuitDesc), P(D), P(I)]),
        "mpdo_batch_run_host": (I, [I, P(VP), I, P(CircuitHostDesc), P(D), P(I)]),
        "mpdo_get_site": (I, [VP, I, P(D), S, P(I)]),
        "mpdo_destroy": (I, [VP]),
        "mpdo_last_error": (C.c_char_p, [VP]),
        "mpdo_build_block_channel": (I, [D, D, D, D, D, D, D, D, P(D), P(D), D, P(D), I, P(I)]),
        "mpdo_build_cz_pulse": (I, [P(Pulse), D, D, D, D, I, P(D), P(D), P(D)]),
        "mpdo_build_crosstalk_cz": (I, [P(Pulse), D, I, P(D)]),
        "mpdo_build_qaoa_layer_cz": (I, [I, I, D, D, D, D, P(D), D, D, P(I), P(I), P(D),
                                         C.c_size_t]),
        "mpdo_build_qaoa_layer": (I, [I, I, D, D, D, D, D, D, D, D, D, D, D, D, P(I), P(I),
                                      P(D), S]),
        "mpdo_build_qaoa_layer_appe": (I, [I, I, D, D, D, D, D, D, D, D, D, D, D, I, D, P(I),
                                           P(I), P(D), S]),
        "mpdo_build_rcs_layer": (I, [I, I, P(D), D, D, D, D, D, D, D, D, P(I), P(I), P(D), S]),
        "mpdo_kernel_launches": (C.c_longlong, []),
        "mpdo_profile": (I, [VP, I]),
        "mpdo_profile_read": (I, [VP, I, P(D), P(C.c_longlong), P(D)]),
        "mpdo_mlp_create": (I, [I, P(I), I, VP, P(VP)]),
        "mpdo_mlp_n_params": (C.c_longlong, [VP]),
        "mpdo_mlp_set_params": (I, [VP, P(C.c_float)]),
        "mpdo_mlp_get_params": (I, [VP, P(C.c_float)]),
        "mpdo_mlp_forward": (I, [VP, I, VP, VP]),
        "mpdo_mlp_loss_grad": (I, [VP, I, VP, VP, P(C.c_float), P(C.c_float)]),
        "mpdo_mlp_adam_step": (I, [VP, C.c_float]),
        "mpdo_mlp_input_grad": (I, [VP, I, VP, P(C.c_float), VP]),
        "mpdo_mlp_destroy": (I, [VP]),
        "mpdo_mlp_set_precision": (I, [VP, I]),
        "mpdo_autotune_gemm": (I, [I, VP, I, P(I)]),
        "mpdo_kernel_cgemm": (I, [I, I, I, I, I, I, VP, C.c_long, C.c_long, VP, C.c_long,
                                  C.c_long, VP, C.c_long, C.c_long, I, VP]),
        "mpdo_kernel_heig": (I, [I, I, VP, VP, P(D), P(I), VP]),
        "mpdo_heig_noalloc": (I, [I, I, VP, VP, P(D), P(I), VP]),
        "mpdo_tc_gemm_launches": (C.c_longlong, []),
        "mpdo_kernel_tcgemm_exact": (I, [I, I, I, I, I, VP, C.c_long, C.c_long, VP, C.c_long,
                                         C.c_long, VP, C.c_long, C.c_long, I, VP]),
        "mpdo_kernel_tcgemm_real": (I, [I, I, I, I, VP, C.c_long, VP, C.c_long, VP, C.c_long,
                                        VP]),
        "mpdo_kernel_tcgemm": (I, [I, I, I, I, I, I, VP, C.c_long, C.c_long, VP, C.c_long,
                                   C.c_long, VP, C.c_long, C.c_long, I, VP]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


LIB = _load()


def _check(rc: int, handle=None):
    if rc != 0:
        msg = LIB.mpdo_last_error(handle)
        raise MpdoError(rc, msg.decode() if msg else "")


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


_CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy: the legacy default stream's handle


def _current_stream():
    """torch's current stream as a cudaStream_t.  torch reports its default stream as 0,
    which the library reads as "create a stream of your own"; it is passed as
    cudaStreamLegacy instead, so library kernels stay ordered with torch's work."""
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream or _CUDA_STREAM_LEGACY)
    except ImportError:
        pass
    return C.c_void_p(None)


# ------------------------------------------------------------------ channels (host, a0)
def build_block_channel(angle_zz: float, gamma_diss: float, gamma_deph: float,
                        xtalk_phase: float = 0.0, delta_pp: float = 0.0, b0: float = 1 / 16,
                        b1: float = 1 / 16, bd: float = 7 / 8, post_left=None, post_right=None,
                        eta: float = 1e-15) -> np.ndarray:
    """Kraus set (M, 9, 9) complex128 of one noisy ZZ block (library channel builder)."""
    out = np.zeros((81, 81, 2))
    m = C.c_int(0)
    pl = None if post_left is None else np.ascontiguousarray(np.asarray(post_left, complex)).view(float)
    pr = None if post_right is None else np.ascontiguousarray(np.asarray(post_right, complex)).view(float)
    rc = LIB.mpdo_build_block_channel(angle_zz, gamma_diss, gamma_deph, xtalk_phase, delta_pp,
                                      b0, b1, bd, None if pl is None else _dptr(pl),
                                      None if pr is None else _dptr(pr), eta, _dptr(out), 81,
                                      C.byref(m))
    _check(rc)
    return out[: m.value].view(complex).reshape(m.value, 9, 9)


def build_qaoa_layer(n_sites: int, k: int, alpha: float, beta: float, J: float = 1.0,
                     bz: float = 0.0, gamma_diss: float = 0.0, gamma_deph: float = 0.0,
                     xtalk_phase: float = 0.0, delta_pp: float = 0.0, b0: float = 1 / 16,
                     b1: float = 1 / 16, bd: float = 7 / 8, eta: float = 1e-15,
                     appe_part: Optional[int] = None):
    """Ordered two-site ops [(site, Kraus (M,9,9))] of QAOA layer k (library builder).
    appe_part 0 / 1: the coherent / incoherent part of the dissipation (App. E)."""
    nops = n_sites - 1
    sites = np.zeros(nops, dtype=np.int32)
    ms = np.zeros(nops, dtype=np.int32)
    cap = nops * 81 * 81
    out = np.zeros((cap, 2))
    sp = sites.ctypes.data_as(C.POINTER(C.c_int))
    mp_ = ms.ctypes.data_as(C.POINTER(C.c_int))
    if appe_part is None:
        rc = LIB.mpdo_build_qaoa_layer(n_sites, k, alpha, beta, J, bz, gamma_diss, gamma_deph,
                                       xtalk_phase, delta_pp, b0, b1, bd, eta, sp, mp_,
                                       _dptr(out), cap)
    else:
        rc = LIB.mpdo_build_qaoa_layer_appe(n_sites, k, alpha, beta, J, bz, gamma_diss,
                                            gamma_deph, xtalk_phase, delta_pp, b0, b1, bd,
                                            int(appe_part), eta, sp, mp_, _dptr(out), cap)
    _check(rc)
    flat = out.view(complex).reshape(-1)
    ops, off = [], 0
    for s, m in zip(sites, ms):
        ops.append((int(s), flat[off: off + m * 81].reshape(m, 9, 9).copy()))
        off += m * 81
    return ops


def build_cz_pulse(gamma_diss: float = 0.0, gamma_deph: float = 0.0, b0: float = 1 / 16,
                   b1: float = 1 / 16, n_steps: int = 2000, pulse: Optional[dict] = None):
    """Pulse-level CZ channel (gate model G1, host builder): (superoperator (81, 81),
    phi_1, noiseless average-gate infidelity).  pulse: dict of Pulse fields (default the
    Gaussian CZ of Fig. 1)."""
    p = Pulse(**(pulse or GAUSSIAN_CZ))
    out = np.zeros((81 * 81, 2))
    phi1, infid = C.c_double(0.0), C.c_double(0.0)
    _check(LIB.mpdo_build_cz_pulse(C.byref(p), gamma_diss, gamma_deph, b0, b1, n_steps,
                                   _dptr(out), C.byref(phi1), C.byref(infid)))
    return out.view(complex).reshape(81, 81).copy(), phi1.value, infid.value


def build_crosstalk_cz(b_x: Optional[float] = None, n_steps: int = 2000,
                       pulse: Optional[dict] = None):
    """Four-site crosstalk CZ (81 x 81 unitary on (i-1, i, i+1, i+2), Sec. III.B, host
    builder): the pulse CZ on (i, i+1) with each active atom's detuning shifted by b_x when
    its non-active neighbour is in |r> (default b_x: the pulse's blockade)."""
    p = Pulse(**(pulse or GAUSSIAN_CZ))
    out = np.zeros((81 * 81, 2))
    _check(LIB.mpdo_build_crosstalk_cz(C.byref(p), p.blockade if b_x is None else b_x, n_steps,
                                       _dptr(out)))
    return out.view(complex).reshape(81, 81).copy()


def build_qaoa_layer_cz(n_sites: int, k: int, alpha: float, beta: float, cz_superop,
                        J: float = 1.0, bz: float = 0.0, xtalk_phase: float = 0.0,
                        eta: float = 1e-15):
    """Ordered two-site ops of QAOA layer k with every CZ replaced by cz_superop (81 x 81)."""
    nops = n_sites - 1
    sites = np.zeros(nops, dtype=np.int32)
    ms = np.zeros(nops, dtype=np.int32)
    cap = nops * 81 * 81
    out = np.zeros((cap, 2))
    scz = np.ascontiguousarray(np.asarray(cz_superop, dtype=complex).reshape(81, 81)).view(float)
    rc = LIB.mpdo_build_qaoa_layer_cz(n_sites, k, alpha, beta, J, bz, _dptr(scz.reshape(-1)),
                                      xtalk_phase, eta,
                                      sites.ctypes.data_as(C.POINTER(C.c_int)),
                                      ms.ctypes.data_as(C.POINTER(C.c_int)), _dptr(out), cap)
    _check(rc)
    flat = out.view(complex).reshape(-1)
    ops, off = [], 0
    for s, m in zip(sites, ms):
        ops.append((int(s), flat[off: off + m * 81].reshape(m, 9, 9).copy()))
        off += m * 81
    return ops


def build_rcs_layer(n_sites: int, k: int, haar, gamma_diss: float = 0.0,
                    gamma_deph: float = 0.0, xtalk_phase: float = 0.0, delta_pp: float = 0.0,
                    b0: float = 1 / 16, b1: float = 1 / 16, bd: float = 7 / 8,
                    eta: float = 1e-15):
    """Ordered two-site ops [(site, Kraus (M,9,9))] of random-circuit layer k (library
    builder); haar: (n_sites, 2, 2) complex one-qubit gates of the layer."""
    nops = n_sites - 1
    sites = np.zeros(nops, dtype=np.int32)
    ms = np.zeros(nops, dtype=np.int32)
    cap = nops * 81 * 81
    out = np.zeros((cap, 2))
    h = np.ascontiguousarray(np.asarray(haar, dtype=complex).reshape(n_sites, 2, 2)).view(float)
    rc = LIB.mpdo_build_rcs_layer(n_sites, k, _dptr(h.reshape(-1)), gamma_diss, gamma_deph,
                                  xtalk_phase, delta_pp, b0, b1, bd, eta,
                                  sites.ctypes.data_as(C.POINTER(C.c_int)),
                                  ms.ctypes.data_as(C.POINTER(C.c_int)), _dptr(out), cap)
    _check(rc)
    flat = out.view(complex).reshape(-1)
    ops, off = [], 0
    for s_, m in zip(sites, ms):
        ops.append((int(s_), flat[off: off + m * 81].reshape(m, 9, 9).copy()))
        off += m * 81
    return ops


def circuit_layers(c, appe_part: Optional[int] = None) -> List[list]:
    """Library-built op lists for every layer of a workload description (synth.Circuit, or
    synth.RcsCircuit for the random circuits).  appe_part (QAOA only): 0 / 1 builds the
    coherent / incoherent part of the dissipation (App. E) instead of the full blocks."""
    if hasattr(c, "haar"):
        return [build_rcs_layer(c.n_sites, k, c.haar[k], c.gamma_diss, c.gamma_deph,
                                c.xtalk_phase, c.delta_pp, c.b0, c.b1, c.bd)
                for k in range(c.depth)]
    return [build_qaoa_layer(c.n_sites, k, c.alpha[k], c.beta[k], c.J, c.bz, c.gamma_diss,
                             c.gamma_deph, c.xtalk_phase, c.delta_pp, c.b0, c.b1, c.bd,
                             appe_part=appe_part)
            for k in range(c.p)]


class _LayerArgs:
    """Keeps the ctypes layer and its arrays alive for one call."""

    def __init__(self, ops):
        self.arrays = []
        self.cops = (Op * max(1, len(ops)))()
        for n, op in enumerate(ops):
            if len(op) == 2:
                site, k = op
                kind = 2
            else:
                kind, site, k = op
            arr = np.ascontiguousarray(np.asarray(k, dtype=complex))
            if kind == 1:
                arr = arr.reshape(1, 3, 3)
            else:
                arr = arr.reshape(-1, 9, 9)
            flat = arr.reshape(-1).view(float)
            self.arrays.append(flat)
            self.cops[n] = Op(kind, int(site), arr.shape[0], _dptr(flat))
        self.layer = Layer(len(ops), self.cops)


class Mpdo:
    """One MPDO on the GPU (handle of libmpdo)."""

    def __init__(self, n_sites: int, chi_max: int, k_max: int, m_max: int = 25,
                 prec: str = "fp64", sv_cutoff: float = 0.0, kraus_cutoff: float = 0.0,
                 use_ppt: bool = True, init_vec: Optional[Sequence[complex]] = None,
                 stream=None, own_stream: bool = False, gram_fp64: bool = False,
                 order: str = "snake", allocator=None):
        """allocator: optional (alloc(bytes) -> device address or 0, free(address)) pair that
        will own every device buffer of the handle (e.g. torch's caching allocator)."""
        self.n = n_sites
        if own_stream:
            st = C.c_void_p(None)            # the library creates a non-blocking stream
        else:
            st = _current_stream() if stream is None else C.c_void_p(stream)
        cfg = Config(n_sites, 3, chi_max, k_max, m_max, PREC[prec], sv_cutoff, kraus_cutoff,
                     int(use_ppt), st, int(gram_fp64), ORDER[order])
        self._hooks = None
        if allocator is not None:
            fa, ff = allocator
            self._hooks = (ALLOC_FN(lambda nbytes, ctx: fa(int(nbytes)) or None),
                           FREE_FN(lambda ptr, ctx: ff(ptr)))
            cfg.alloc, cfg.free = self._hooks
        self._h = C.c_void_p(None)
        v = None if init_vec is None else np.ascontiguousarray(np.asarray(init_vec, complex)).view(float)
        rc = LIB.mpdo_create(C.byref(cfg), None if v is None else _dptr(v), C.byref(self._h))
        _check(rc)
        self.prec = prec

    def close(self):
        if self._h:
            LIB.mpdo_destroy(self._h)
            self._h = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, init_vec=None):
        v = None if init_vec is None else np.ascontiguousarray(np.asarray(init_vec, complex)).view(float)
        _check(LIB.mpdo_reset(self._h, None if v is None else _dptr(v)), self._h)

    def apply_layer(self, ops) -> dict:
        args = _LayerArgs(ops)
        st = TruncStats()
        _check(LIB.mpdo_apply_layer(self._h, C.byref(args.layer), C.byref(st)), self._h)
        return st.as_dict()

    def upload_layer(self, ops):
        args = _LayerArgs(ops)
        dl = C.c_void_p(None)
        _check(LIB.mpdo_layer_upload(self._h, C.byref(args.layer), C.byref(dl)), self._h)
        return dl

    def apply_uploaded(self, dl) -> dict:
        st = TruncStats()
        _check(LIB.mpdo_apply_dlayer(self._h, dl, C.byref(st)), self._h)
        return st.as_dict()

    def free_uploaded(self, dl):
        _check(LIB.mpdo_layer_free(self._h, dl), self._h)

    def truncate(self, chi_max: int, k_max: int, use_ppt: bool = True) -> dict:
        st = TruncStats()
        _check(LIB.mpdo_truncate(self._h, chi_max, k_max, int(use_ppt), C.byref(st)), self._h)
        return st.as_dict()

    def expect_energy(self, J: float = 1.0, hx: float = 1.0, bz: float = 0.0) -> dict:
        vals = [C.c_double() for _ in range(4)]
        _check(LIB.mpdo_expect_energy(self._h, J, hx, bz, *[C.byref(v) for v in vals]),
               self._h)
        return dict(zip(("e_raw", "e_succ", "p_succ", "trace"), (v.value for v in vals)))

    def second_order(self, cut: int) -> dict:
        """xi = tr rho^2 / (tr rho)^2, collision probability, Renyi-2 entropies of the two
        halves at `cut` and their mutual information (library environments)."""
        v = [C.c_double(0) for _ in range(5)]
        _check(LIB.mpdo_expect_second_order(self._h, cut, *[C.byref(x) for x in v]), self._h)
        return dict(zip(("xi", "collision", "s2_left", "s2_right", "i2"), [x.value for x in v]))

    def sample_probs(self, n_samples: int, seed: int) -> Tuple[np.ndarray, np.ndarray]:
        bits = np.zeros((n_samples, self.n), dtype=np.uint8)
        probs = np.zeros(n_samples)
        _check(LIB.mpdo_sample_probs(self._h, n_samples, seed,
                                     bits.ctypes.data_as(C.POINTER(C.c_uint8)), _dptr(probs)),
               self._h)
        return bits, probs

    def reconfigure(self, n_sites: int, chi_max: int, k_max: int, use_ppt: bool = True):
        _check(LIB.mpdo_reconfigure(self._h, n_sites, chi_max, k_max, int(use_ppt), None),
               self._h)
        self.n = n_sites

    def profile(self, class_mask: int):
        """Time launches of the selected kernel classes with CUDA events (bit 0: GEMMs,
        bit 1: eigensolver, bit 2: other kernels); 0 switches it off."""
        _check(LIB.mpdo_profile(self._h, class_mask), self._h)

    def profile_read(self, cls: int) -> dict:
        ms, n, fl = C.c_double(), C.c_longlong(), C.c_double()
        _check(LIB.mpdo_profile_read(self._h, cls, C.byref(ms), C.byref(n), C.byref(fl)),
               self._h)
        return dict(ms=ms.value, launches=n.value, flops=fl.value)

    def dims(self):
        b = np.zeros(self.n - 1, dtype=np.int32)
        k = np.zeros(self.n, dtype=np.int32)
        c = C.c_int(0)
        _check(LIB.mpdo_get_dims(self._h, b.ctypes.data_as(C.POINTER(C.c_int)),
                                 k.ctypes.data_as(C.POINTER(C.c_int)), C.byref(c)), self._h)
        return b, k, c.value

    def site(self, n: int) -> np.ndarray:
        b, k, _ = self.dims()
        dl = 1 if n == 0 else int(b[n - 1])
        dr = 1 if n == self.n - 1 else int(b[n])
        cap = dl * 3 * int(k[n]) * dr
        out = np.zeros(2 * cap)
        dims = (C.c_int * 4)()
        _check(LIB.mpdo_get_site(self._h, n, _dptr(out), cap, dims), self._h)
        return out.view(complex).reshape(tuple(dims))


def batch_run(pool: Sequence["Mpdo"], circuits: Sequence[dict]) -> np.ndarray:
    """Run circuits concurrently on a pool of handles (one stream and host thread each).

    circuits: dicts with n_sites, chi_max, k_max, layers (uploaded with pool[0].upload_layer),
    and optionally use_ppt, J, hx, b.  Returns an (n, 4) array of e_raw, e_succ, p_succ, trace.
    """
    handles = (C.c_void_p * len(pool))(*[m._h.value for m in pool])
    descs = (CircuitDesc * max(1, len(circuits)))()
    keep = []
    for i, c in enumerate(circuits):
        arr = (C.c_void_p * max(1, len(c["layers"])))(*[dl.value for dl in c["layers"]])
        keep.append(arr)
        descs[i] = CircuitDesc(c["n_sites"], c["chi_max"], c["k_max"], int(c.get("use_ppt", True)),
                               len(c["layers"]), arr, c.get("J", 1.0), c.get("hx", 1.0),
                               c.get("b", 0.0))
    out = np.zeros((len(circuits), 4))
    status = np.zeros(len(circuits), dtype=np.int32)
    rc = LIB.mpdo_batch_run(len(pool), handles, len(circuits), descs, _dptr(out),
                            status.ctypes.data_as(C.POINTER(C.c_int)))
    if rc != 0:
        bad = [(i, int(x)) for i, x in enumerate(status) if x]
        msg = LIB.mpdo_last_error(None)
        raise MpdoError(rc, f"{msg.decode() if msg else ''}; failed circuits {bad[:8]}")
    return out


class HostCircuit:
    """A circuit's layers marshalled once into the C ABI's host layout (host memory), for
    batch_run_host: n_sites, chi_max, k_max, layers (op lists as for Mpdo.apply_layer),
    use_ppt, J, hx, b."""

    def __init__(self, n_sites: int, chi_max: int, k_max: int, layers, use_ppt: bool = True,
                 J: float = 1.0, hx: float = 1.0, b: float = 0.0):
        self._args = [_LayerArgs(ops) for ops in layers]
        self._layers = (Layer * max(1, len(self._args)))(*[a.layer for a in self._args])
        self.desc = CircuitHostDesc(n_sites, chi_max, k_max, int(use_ppt), len(self._args),
                                    self._layers, J, hx, b)


def batch_run_host(pool: Sequence["Mpdo"], circuits: Sequence[HostCircuit]) -> np.ndarray:
    """batch_run for circuits held in host memory: each worker uploads its circuit's layers
    on its own stream.  Returns an (n, 4) array of e_raw, e_succ, p_succ, trace."""
    handles = (C.c_void_p * len(pool))(*[m._h.value for m in pool])
    descs = (CircuitHostDesc * max(1, len(circuits)))(*[c.desc for c in circuits])
    out = np.zeros((len(circuits), 4))
    status = np.zeros(len(circuits), dtype=np.int32)
    rc = LIB.mpdo_batch_run_host(len(pool), handles, len(circuits), descs, _dptr(out),
                                 status.ctypes.data_as(C.POINTER(C.c_int)))
    if rc != 0:
        bad = [(i, int(x)) for i, x in enumerate(status) if x]
        msg = LIB.mpdo_last_error(None)
        raise MpdoError(rc, f"{msg.decode() if msg else ''}; failed circuits {bad[:8]}")
    return out


class Mlp:
    """MLP surrogate on the GPU (tanh hidden layers, linear output): FP32, or BF16 tensor-core
    products with FP32 accumulation and parameters."""

    def __init__(self, widths: Sequence[int], max_batch: int, stream=None, bf16: bool = False):
        """stream: CUDA stream for the network's kernels; default torch's current stream,
        so device inputs written by torch are ordered before the network reads them.
        bf16: products on the tensor cores with BF16 operands (FP32 accumulation and FP32
        master parameters)."""
        arr = (C.c_int * len(widths))(*widths)
        self._h = C.c_void_p(None)
        st = _current_stream() if stream is None else C.c_void_p(stream)
        _check(LIB.mpdo_mlp_create(len(widths) - 1, arr, max_batch, st, C.byref(self._h)))
        self.widths = list(widths)
        self.n_params = int(LIB.mpdo_mlp_n_params(self._h))
        if bf16:
            _check(LIB.mpdo_mlp_set_precision(self._h, 1))

    def close(self):
        if self._h:
            LIB.mpdo_mlp_destroy(self._h)
            self._h = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _fptr(a):
        return a.ctypes.data_as(C.POINTER(C.c_float))

    def set_params(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.n_params
        _check(LIB.mpdo_mlp_set_params(self._h, self._fptr(flat)))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(LIB.mpdo_mlp_get_params(self._h, self._fptr(out)))
        return out

    def forward(self, x, y):
        _check(LIB.mpdo_mlp_forward(self._h, x.shape[0], C.c_void_p(x.data_ptr()),
                                    C.c_void_p(y.data_ptr())))

    def loss_grad(self, x, t, want_grad: bool = False):
        loss = C.c_float(0)
        g = np.zeros(self.n_params, dtype=np.float32) if want_grad else None
        _check(LIB.mpdo_mlp_loss_grad(self._h, x.shape[0], C.c_void_p(x.data_ptr()),
                                      C.c_void_p(t.data_ptr()), C.byref(loss),
                                      None if g is None else self._fptr(g)))
        return loss.value, g

    def adam_step(self, lr: float):
        _check(LIB.mpdo_mlp_adam_step(self._h, lr))

    def input_grad(self, x, wout, gx):
        w = np.ascontiguousarray(wout, dtype=np.float32)
        _check(LIB.mpdo_mlp_input_grad(self._h, x.shape[0], C.c_void_p(x.data_ptr()),
                                       self._fptr(w), C.c_void_p(gx.data_ptr())))


def mlp_flat(params) -> np.ndarray:
    """[(W_l, b_l)] -> the flat parameter layout of the library."""
    return np.concatenate([np.concatenate([w.reshape(-1), b.reshape(-1)]) for w, b in params])


def mlp_unflat(flat, widths):
    out, off = [], 0
    for a, b in zip(widths[:-1], widths[1:]):
        w = flat[off: off + a * b].reshape(a, b)
        off += a * b
        bb = flat[off: off + b]
        off += b
        out.append((w, bb))
    return out


def kernel_launches() -> int:
    """Kernels launched by libmpdo in this process so far."""
    return int(LIB.mpdo_kernel_launches())


# ------------------------------------------------------ kernel-level entry points (tests)
def autotune_gemm(prec: int, reps: int = 3, stream=None) -> int:
    """Tile-shape autotuner of the complex GEMMs (prec 0: FP64 products, 1: FP32); reps <= 0
    resets to the built-in size rules.  Returns the number of buckets tuned."""
    st = _current_stream() if stream is None else C.c_void_p(stream)
    n = C.c_int(0)
    _check(LIB.mpdo_autotune_gemm(prec, st, reps, C.byref(n)))
    return n.value


def kernel_cgemm(prec: int, opa: int, opb: int, m: int, n: int, k: int, a, lda: int, sa: int,
                 b, ldb: int, sb: int, c, ldc: int, sc: int, batch: int, stream=None):
    """c = op(a) op(b) on device tensors (complex128 if prec == 0 else complex64)."""
    st = _current_stream() if stream is None else C.c_void_p(stream)
    _check(LIB.mpdo_kernel_cgemm(prec, opa, opb, m, n, k, C.c_void_p(a.data_ptr()), lda, sa,
                                 C.c_void_p(b.data_ptr()), ldb, sb, C.c_void_p(c.data_ptr()),
                                 ldc, sc, batch, st))


def kernel_heig(prec: int, n: int, a, v, w, stream=None) -> int:
    """Hermitian eigendecomposition of the device matrix a (n x n) -> w (desc), v."""
    st = _current_stream() if stream is None else C.c_void_p(stream)
    sweeps = C.c_int(0)
    _check(LIB.mpdo_kernel_heig(prec, n, C.c_void_p(a.data_ptr()), C.c_void_p(v.data_ptr()),
                                C.cast(C.c_void_p(w.data_ptr()), C.POINTER(C.c_double)),
                                C.byref(sweeps), st))
    return sweeps.value


HEIG_NOALLOC_NMAX = 192


def kernel_heig_noalloc(prec: int, n: int, a, v, w, stream=None) -> int:
    """Allocation-free eigensolver entry point (scratch in a fixed device array, n <= 192)."""
    st = _current_stream() if stream is None else C.c_void_p(stream)
    sweeps = C.c_int(0)
    _check(LIB.mpdo_heig_noalloc(prec, n, C.c_void_p(a.data_ptr()), C.c_void_p(v.data_ptr()),
                                 C.cast(C.c_void_p(w.data_ptr()), C.POINTER(C.c_double)),
                                 C.byref(sweeps), st))
    return sweeps.value


TC_MODES = {"tf32": 0, "tf32x3": 1, "bf16": 2, "bf16x3": 3}


def tc_gemm_launches() -> int:
    """Tensor-core (tcgen05) GEMM kernels launched by libmpdo in this process so far."""
    return int(LIB.mpdo_tc_gemm_launches())


def kernel_tcgemm_real(elt: int, m: int, n: int, k: int, a, lda: int, b, ldb: int, d, ldd: int,
                       stream=None):
    """d (m x n, FP32) = a (m x k) b (n x k)^T on the tensor cores; a, b FP32 (read as TF32,
    elt 4) or BF16 (elt 2) device tensors, K-major."""
    st = _current_stream() if stream is None else C.c_void_p(stream)
    _check(LIB.mpdo_kernel_tcgemm_real(elt, m, n, k, C.c_void_p(a.data_ptr()), lda,
                                       C.c_void_p(b.data_ptr()), ldb, C.c_void_p(d.data_ptr()),
                                       ldd, st))


def kernel_tcgemm(mode, opa: int, opb: int, m: int, n: int, k: int, a, lda: int, sa: int, b,
                  ldb: int, sb: int, c, ldc: int, sc: int, batch: int, stream=None):
    """c = op(a) op(b) (complex64 device tensors) on the tensor cores in mode "tf32",
    "tf32x3", "bf16" or "bf16x3"."""
    st = _current_stream() if stream is None else C.c_void_p(stream)
    md = TC_MODES[mode] if isinstance(mode, str) else int(mode)
    _check(LIB.mpdo_kernel_tcgemm(md, opa, opb, m, n, k, C.c_void_p(a.data_ptr()), lda, sa,
                                  C.c_void_p(b.data_ptr()), ldb, sb, C.c_void_p(c.data_ptr()),
                                  ldc, sc, batch, st))


def kernel_tcgemm_exact(opa: int, opb: int, m: int, n: int, k: int, a, lda: int, sa: int, b,
                        ldb: int, sb: int, c, ldc: int, sc: int, batch: int, stream=None):
    """c (complex128) = op(a) op(b) for complex64 device tensors a, b: FP64-accurate exact
    slice products on the BF16 tensor cores."""
    st = _current_stream() if stream is None else C.c_void_p(stream)
    _check(LIB.mpdo_kernel_tcgemm_exact(opa, opb, m, n, k, C.c_void_p(a.data_ptr()), lda, sa,
                                        C.c_void_p(b.data_ptr()), ldb, sb,
                                        C.c_void_p(c.data_ptr()), ldc, sc, batch, st))


class Vmpo:
    """Vectorized-MPO engine on the GPU (rho as an MPS over (s, s'), PPT on the bond)."""

    def __init__(self, n_sites: int, chi_max: int, ppt: bool = True, sv_cutoff: float = 0.0,
                 init_vec: Optional[Sequence[complex]] = None, stream=None, tc: bool = False):
        self.n = n_sites
        st = C.c_void_p(None) if stream is None else C.c_void_p(stream)
        v = None if init_vec is None else np.ascontiguousarray(np.asarray(init_vec, complex)).view(float)
        self._h = C.c_void_p(None)
        _check(LIB.mpdo_vmpo_create(n_sites, chi_max, int(ppt), sv_cutoff,
                                    None if v is None else _dptr(v), st, C.byref(self._h)))
        if tc:
            self.set_precision(1)

    def set_precision(self, mode: int):
        """0: FP64 CUDA cores and Jacobi; 1: exact-slice tensor-core products and the mixed
        eigensolver."""
        _check(LIB.mpdo_vmpo_set_precision(self._h, mode))

    def close(self):
        if self._h:
            LIB.mpdo_vmpo_destroy(self._h)
            self._h = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_layer(self, ops) -> dict:
        lay = _LayerArgs(ops)
        st = TruncStats()
        _check(LIB.mpdo_vmpo_apply_layer(self._h, C.byref(lay.layer), C.byref(st)))
        return st.as_dict()

    def expect_energy(self, J: float = 1.0, hx: float = 1.0, bz: float = 0.0) -> dict:
        v = [C.c_double(0) for _ in range(4)]
        _check(LIB.mpdo_vmpo_expect_energy(self._h, J, hx, bz, *[C.byref(x) for x in v]))
        return dict(zip(("e_raw", "e_succ", "p_succ", "trace"), [x.value for x in v]))

    def purity(self) -> float:
        p = C.c_double(0)
        _check(LIB.mpdo_vmpo_purity(self._h, C.byref(p)))
        return p.value

    def collision(self) -> float:
        """sum_x <x|rho|x>^2 / (tr rho)^2."""
        z = C.c_double(0)
        _check(LIB.mpdo_vmpo_collision(self._h, C.byref(z)))
        return z.value

    def dims(self):
        b = np.zeros(self.n - 1, dtype=np.int32)
        c = C.c_int(0)
        _check(LIB.mpdo_vmpo_get_dims(self._h, b.ctypes.data_as(C.POINTER(C.c_int)), C.byref(c)))
        return b, c.value
