"""GB300-native commutator-free exponential time-propagator (CFET) with a
device Lanczos/Krylov exponential, after Alvermann & Fehske, arXiv:1102.5071.

This module is the thin Python binding of the C ABI declared in
``include/cfet.h``: it marshals arguments (torch tensors for device memory and
streams, Python callables for the drives) and calls the compiled library.
Every step of the propagation runs in the library's CUDA kernels; there is no
CPU path, and a missing library or device raises.
"""

from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _capi
from ._capi import SCHEME_IDS, STATUS_NAMES


class CfetError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


# ---------------------------------------------------------------- operators
@dataclass
class XXZChain:
    """H0 = sum_i [J (X_i X_{i+1} + Y_i Y_{i+1}) + J Delta Z_i Z_{i+1}] + sum_i h_i Z_i (open chain)."""
    N: int
    J: float
    Delta: float
    h: np.ndarray


@dataclass
class XField:
    """V = sum_i a_i X_i."""
    N: int
    a: np.ndarray


class PauliSum:
    """P = sum_t c_t S_t on a chain of N spins, every S_t a tensor product of
    X, Y, Z on some sites (a Pauli string).  terms: (c, label) pairs with label
    a string over 'IXYZ' whose character i acts on site i (site 0 first), or a
    dict {site: 'X' | 'Y' | 'Z'}.  Passed to the library as X and Z bit masks
    with Y_i = i X_i Z_i (the phase i^popc(x & z) of the C ABI)."""

    def __init__(self, N, terms):
        self.N = int(N)
        xs, zs, cs = [], [], []
        for c, label in terms:
            ops = dict(enumerate(label)) if isinstance(label, str) else dict(label)
            x = z = 0
            for site, letter in ops.items():
                site = int(site)
                if not 0 <= site < self.N:
                    raise ValueError(f"site {site} outside the chain of {self.N}")
                letter = letter.upper()
                if letter in ("X", "Y"):
                    x |= 1 << site
                if letter in ("Z", "Y"):
                    z |= 1 << site
                if letter not in ("I", "X", "Y", "Z"):
                    raise ValueError(f"unknown Pauli letter {letter!r}")
            xs.append(x)
            zs.append(z)
            cs.append(float(c))
        self.xmask = np.array(xs, dtype=np.uint64)
        self.zmask = np.array(zs, dtype=np.uint64)
        self.coeff = np.array(cs, dtype=np.float64)


@dataclass
class DIA:
    """(D v)[r] = sum_d values[d, r] v[r + offsets[d]] (real, symmetric)."""
    offsets: np.ndarray
    values: np.ndarray


class CSR:
    """Hermitian sparse operator in compressed sparse row form:
    (A v)[r] = sum_{e in [row_ptr[r], row_ptr[r+1])} values[e] v[col_idx[e]];
    values real (a real symmetric operator) or complex.  from_scipy() takes
    any scipy.sparse matrix."""

    def __init__(self, row_ptr, col_idx, values):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        v = np.asarray(values)
        self.re = np.ascontiguousarray(v.real, dtype=np.float64)
        self.im = np.ascontiguousarray(v.imag, dtype=np.float64) if np.iscomplexobj(v) else None
        self.dim = len(self.row_ptr) - 1

    @classmethod
    def from_scipy(cls, m):
        m = m.tocsr()
        return cls(m.indptr, m.indices, m.data)


def _op_struct(op, keep):
    s = _capi.cfet_op()
    if isinstance(op, XXZChain):
        h = np.ascontiguousarray(op.h, dtype=np.float64)
        keep.append(h)
        s.kind, s.nsites, s.dim = _capi.CFET_OP_XXZ_CHAIN, op.N, 1 << op.N
        s.J, s.Delta = op.J, op.Delta
        s.site_coeff = h.ctypes.data_as(_capi.c_double_p)
    elif isinstance(op, XField):
        a = np.ascontiguousarray(op.a, dtype=np.float64)
        keep.append(a)
        s.kind, s.nsites, s.dim = _capi.CFET_OP_X_FIELD, op.N, 1 << op.N
        s.site_coeff = a.ctypes.data_as(_capi.c_double_p)
    elif isinstance(op, DIA):
        off = np.ascontiguousarray(op.offsets, dtype=np.int64)
        val = np.ascontiguousarray(op.values, dtype=np.float64)
        keep += [off, val]
        s.kind, s.dim, s.ndiag = _capi.CFET_OP_DIA, val.shape[1], val.shape[0]
        s.offsets = off.ctypes.data_as(_capi.c_int64_p)
        s.values = val.ctypes.data_as(_capi.c_double_p)
    elif isinstance(op, PauliSum):
        xm, zm, c = (np.ascontiguousarray(a) for a in (op.xmask, op.zmask, op.coeff))
        keep += [xm, zm, c]
        s.kind, s.nsites, s.dim, s.nterms = _capi.CFET_OP_PAULI, op.N, 1 << op.N, len(c)
        s.xmask = xm.ctypes.data_as(_capi.c_uint64_p)
        s.zmask = zm.ctypes.data_as(_capi.c_uint64_p)
        s.coeff = c.ctypes.data_as(_capi.c_double_p)
    elif isinstance(op, CSR):
        keep += [op.row_ptr, op.col_idx, op.re] + ([op.im] if op.im is not None else [])
        s.kind, s.dim = _capi.CFET_OP_CSR, op.dim
        s.row_ptr = op.row_ptr.ctypes.data_as(_capi.c_int64_p)
        s.col_idx = op.col_idx.ctypes.data_as(_capi.c_int32_p)
        s.csr_re = op.re.ctypes.data_as(_capi.c_double_p)
        s.csr_im = op.im.ctypes.data_as(_capi.c_double_p) if op.im is not None else None
    else:
        raise TypeError(f"unsupported operator {type(op).__name__}")
    return s


def scheme_info(name_or_id):
    """(order, s, M, f[s,M], x[M], w[M], g[s,M]) as used by the device path."""
    lib = _capi.load()
    sid = SCHEME_IDS[name_or_id] if isinstance(name_or_id, str) else int(name_or_id)
    cap = 11 * 4
    f, g = np.zeros(cap), np.zeros(cap)
    x, w = np.zeros(4), np.zeros(4)
    order, s, M = C.c_int32(), C.c_int32(), C.c_int32()
    P = _capi.c_double_p
    st = lib.cfet_scheme_info(sid, C.byref(order), C.byref(s), C.byref(M), f.ctypes.data_as(P),
                              x.ctypes.data_as(P), w.ctypes.data_as(P), g.ctypes.data_as(P), cap)
    if st != 0:
        raise CfetError(st, "unknown scheme")
    s_, M_ = s.value, M.value
    return order.value, s_, M_, f[: s_ * M_].reshape(s_, M_), x[:M_].copy(), w[:M_].copy(), g[: s_ * M_].reshape(s_, M_)


def chebyshev_coefficients(z, tol):
    """(r[0..K], K, tail) of the Chebyshev expansion of exp(-i z x) on [-1, 1]
    used by the CFET_EXPM_CHEBYSHEV path: r_k = (2 - delta_k0) J_k(z), K the
    smallest order whose Bessel tail bound 2 sum_{k>K} |J_k(z)| is <= tol."""
    lib = _capi.load()
    K, tail = C.c_int32(), C.c_double()
    st = lib.cfet_chebyshev_coefficients(float(z), float(tol), 0, None, C.byref(K), C.byref(tail))
    if st != 0:
        raise CfetError(st, "invalid Chebyshev argument")
    r = np.zeros(K.value + 1)
    st = lib.cfet_chebyshev_coefficients(float(z), float(tol), len(r), r.ctypes.data_as(_capi.c_double_p),
                                         C.byref(K), C.byref(tail))
    if st != 0:
        raise CfetError(st, "invalid Chebyshev argument")
    return r, K.value, tail.value


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def probe_copy_gbs(a, b, reps=100, stream=None):
    """Copy rate in GB/s (read + write) of `reps` alternating copies between
    the CUDA tensors a and b (same number of bytes, overwritten) inside one
    launch: the L2-served rate when both fit in L2, the DRAM rate otherwise."""
    import torch
    if not (isinstance(a, torch.Tensor) and isinstance(b, torch.Tensor) and a.is_cuda and b.is_cuda):
        raise TypeError("a and b must be CUDA tensors")
    nbytes = a.numel() * a.element_size()
    if b.numel() * b.element_size() != nbytes or not (a.is_contiguous() and b.is_contiguous()):
        raise ValueError("a and b must be contiguous with the same number of bytes")
    lib = _capi.load()
    out = C.c_double(0.0)
    st = lib.cfet_probe_copy_gbs(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), nbytes, int(reps),
                                 _stream_handle(stream), C.byref(out))
    if st != 0:
        raise CfetError(st, lib.cfet_last_error(None).decode())
    return out.value


def _check_vec(t, dim, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA complex128 tensor")
    if not t.is_contiguous() or t.numel() != dim:
        raise ValueError(f"{name} must be contiguous with {dim} elements")


class Propagator:
    """CFET propagator for H(t) = H0 + sum_k f_k(t) V_k on the current CUDA device.

    H0, V: XXZChain / XField, DIA, CSR or PauliSum operators (see include/cfet.h);
    drives: one callable f_k(t) per V_k.  precision: "default" (fixed point;
    FP64 when a PauliSum is involved), "fx", "f64" or "c64"; expm: "krylov" or
    "chebyshev" (fixed point); picture: "schroedinger" or "interaction" (FP64
    chains); reorth: full re-orthogonalisation of the Lanczos vectors (FP64);
    apply_form: "auto", "elementwise" or "tiled" (XXZ chains in the fixed-point
    and complex64 kernels).
    """

    def __init__(self, H0, V=(), drives=(), *, m_max=16, m_min=2, max_substeps=64, block_size=0,
                 grid_size=0, steps_per_launch=256, barrier_timeout_s=2.0, precision="default", expm="krylov",
                 picture="schroedinger", reorth=False, apply_form="auto"):
        lib = _capi.load()
        V = list(V)
        drives = list(drives)
        if len(V) != len(drives):
            raise ValueError("one drive per drive operator")
        self._keep = []
        h0 = _op_struct(H0, self._keep)
        varr = (_capi.cfet_op * max(1, len(V)))(*[_op_struct(v, self._keep) for v in V])
        self._cbs = [_capi.DRIVE_FN(lambda t, u, fn=fn: float(fn(t))) for fn in drives]
        fns = (_capi.DRIVE_FN * max(1, len(V)))(*self._cbs)
        opt = _capi.cfet_options()
        lib.cfet_options_default(C.byref(opt))
        opt.m_max, opt.m_min, opt.max_substeps = m_max, m_min, max_substeps
        opt.block_size, opt.grid_size, opt.steps_per_launch = block_size, grid_size, steps_per_launch
        opt.barrier_timeout_s = barrier_timeout_s
        opt.precision = _capi.PRECISIONS[precision]
        opt.expm = _capi.EXPM[expm]
        opt.picture = _capi.PICTURES[picture]
        opt.reorth = 1 if reorth else 0
        opt.apply_form = _capi.APPLY_FORMS[apply_form]
        ctx = C.c_void_p()
        st = lib.cfet_create(C.byref(ctx), C.byref(h0), len(V), varr, fns, None, C.byref(opt))
        if st != 0:
            raise CfetError(st, lib.cfet_last_error(None).decode())
        self._lib = lib
        self._ctx = ctx
        self.dim = int(lib.cfet_dim(ctx))
        self.nV = len(V)
        self.m_max = m_max
        self.max_substeps = max_substeps

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.cfet_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, st):
        if st != 0:
            raise CfetError(st, self._lib.cfet_last_error(self._ctx).decode())

    def _coefs(self, c):
        c = np.ascontiguousarray(c, dtype=np.float64)
        if c.shape != (1 + self.nV,):
            raise ValueError(f"expected {1 + self.nV} stage scalars")
        return c

    def apply(self, c, v_in, v_out, stream=None):
        """v_out = (c[0] H0 + sum_k c[1+k] V_k) v_in on the device."""
        c = self._coefs(c)
        _check_vec(v_in, self.dim, "v_in")
        _check_vec(v_out, self.dim, "v_out")
        self._raise(self._lib.cfet_apply(self._ctx, c.ctypes.data_as(_capi.c_double_p), C.c_void_p(v_in.data_ptr()),
                                         C.c_void_p(v_out.data_ptr()), _stream_handle(stream)))

    def expv(self, c, tau, psi, tol, stream=None):
        """psi <- exp(-i tau (c[0] H0 + sum_k c[1+k] V_k)) psi; returns stats."""
        c = self._coefs(c)
        _check_vec(psi, self.dim, "psi")
        stats = _capi.cfet_stats()
        self._raise(self._lib.cfet_expv(self._ctx, c.ctypes.data_as(_capi.c_double_p), float(tau),
                                        C.c_void_p(psi.data_ptr()), float(tol), _stream_handle(stream),
                                        C.byref(stats)))
        return stats.as_dict()

    def propagate(self, psi, t0, dt, nsteps, order=4, tol=1e-10, scheme=None, stream=None, stats=True,
                  forced=None, record=False, record_cap=None):
        """nsteps CFET steps on the device tensor psi (in place).

        forced: decision log to replay, a list over stage exponentials of
        lists of (k, h).  record: return the device's decision log as well.
        Returns stats (dict) or (stats, log) when record is true.
        """
        _check_vec(psi, self.dim, "psi")
        sid = 0 if scheme is None else (SCHEME_IDS[scheme] if isinstance(scheme, str) else int(scheme))
        if scheme is not None:
            order = scheme_info(sid)[0]
        default_ids = {2: 1, 4: 2, 6: 10, 8: 12}
        if sid:
            s = scheme_info(sid)[1]
        elif order in default_ids:
            s = scheme_info(default_ids[order])[1]
        else:
            s = 1   # invalid order: the library rejects the call with CFET_EINVAL
        nexp = int(nsteps) * s
        keep = []
        fd = None
        if forced is not None:
            if len(forced) != nexp:
                raise ValueError("forced log must cover nsteps * s exponentials")
            nsub = np.array([len(x) for x in forced], dtype=np.int32)
            ks = np.array([k for x in forced for k, _ in x], dtype=np.int32)
            hs = np.array([h for x in forced for _, h in x], dtype=np.int32)
            keep += [nsub, ks, hs]
            fd = _capi.cfet_decisions(nexp, nsub.ctypes.data_as(_capi.c_int32_p), ks.ctypes.data_as(_capi.c_int32_p),
                                      hs.ctypes.data_as(_capi.c_int32_p), len(ks), len(ks))
        rd = None
        if record:
            cap = record_cap or max(1, nexp * self.max_substeps)
            rn = np.zeros(nexp, dtype=np.int32)
            rk = np.zeros(cap, dtype=np.int32)
            rh = np.zeros(cap, dtype=np.int32)
            keep += [rn, rk, rh]
            rd = _capi.cfet_decisions(nexp, rn.ctypes.data_as(_capi.c_int32_p), rk.ctypes.data_as(_capi.c_int32_p),
                                      rh.ctypes.data_as(_capi.c_int32_p), cap, 0)
        st_struct = _capi.cfet_stats() if (stats or record) else None
        st = self._lib.cfet_propagate_ex(self._ctx, C.c_void_p(psi.data_ptr()), float(t0), float(dt), int(nsteps),
                                         int(order), sid, float(tol), _stream_handle(stream),
                                         C.byref(fd) if fd is not None else None,
                                         C.byref(rd) if rd is not None else None,
                                         C.byref(st_struct) if st_struct is not None else None)
        self._raise(st)
        out = st_struct.as_dict() if st_struct is not None else None
        if record:
            log, pos = [], 0
            for e in range(nexp):
                n = int(rn[e])
                log.append([(int(rk[pos + i]), int(rh[pos + i])) for i in range(n)])
                pos += n
            return out, log
        return out

    def propagate_host(self, psi_host, t0, dt, nsteps, order=4, tol=1e-10, stream=None):
        """End-to-end form: psi_host (numpy complex128, or a pinned CPU tensor) is
        copied to the device, propagated and copied back in place."""
        if isinstance(psi_host, np.ndarray):
            if psi_host.dtype != np.complex128 or not psi_host.flags.c_contiguous or psi_host.size != self.dim:
                raise ValueError("psi_host must be a contiguous complex128 array of length dim")
            ptr = psi_host.ctypes.data
        else:
            if psi_host.is_cuda or psi_host.numel() != self.dim:
                raise ValueError("psi_host must be a host tensor of length dim")
            ptr = psi_host.data_ptr()
        stats = _capi.cfet_stats()
        self._raise(self._lib.cfet_propagate_host(self._ctx, C.c_void_p(ptr), float(t0), float(dt), int(nsteps),
                                                  int(order), float(tol), _stream_handle(stream), C.byref(stats)))
        return stats.as_dict()

    def kernel_time_ms(self):
        """Device time of the persistent-kernel launches of the last propagate call."""
        ms = C.c_float()
        self._raise(self._lib.cfet_kernel_time_ms(self._ctx, C.byref(ms)))
        return float(ms.value)

    def fidelity_grad(self, psi0, phi, t0, dt, nsteps, amps, omega, phase=0.0, order=4, tol=1e-10,
                      checkpoint_every=None, stream=None):
        """L = 1 - |<phi|psi(T)>|^2 and dL/dA for the single X-field drive
        replaced by f(t) = amps[k] cos(omega t + phase) on segment k (see
        cfet_fidelity_grad).  Returns (loss, grad ndarray, stats dict)."""
        _check_vec(psi0, self.dim, "psi0")
        _check_vec(phi, self.dim, "phi")
        a = np.ascontiguousarray(amps, dtype=np.float64)
        g = np.zeros(a.size)
        loss = C.c_double()
        gs = _capi.cfet_grad_stats()
        ce = int(checkpoint_every) if checkpoint_every else max(1, int(nsteps) // max(1, a.size))
        self._raise(self._lib.cfet_fidelity_grad(
            self._ctx, C.c_void_p(psi0.data_ptr()), C.c_void_p(phi.data_ptr()), float(t0), float(dt), int(nsteps),
            int(order), float(tol), a.size, a.ctypes.data_as(_capi.c_double_p), float(omega), float(phase), ce,
            _stream_handle(stream), C.byref(loss), g.ctypes.data_as(_capi.c_double_p), C.byref(gs)))
        stats = {f: getattr(gs, f) for f, _ in gs._fields_}
        return loss.value, g, stats

    # -------------------------------------------------- time-step selection (Sec. 6.6)
    @staticmethod
    def _sid(scheme):
        return 0 if scheme is None else (SCHEME_IDS[scheme] if isinstance(scheme, str) else int(scheme))

    def error_constant(self, psi0, t0, T, n1, order=4, tol=1e-10, scheme=None, ratio=2.0, stream=None):
        """Error constant c of eps = c T dt^N from runs with n1 and
        round(n1 ratio^(1/N)) steps over [t0, t0 + T]; returns (c, diff, dt2)."""
        _check_vec(psi0, self.dim, "psi0")
        c, d, h2 = C.c_double(), C.c_double(), C.c_double()
        self._raise(self._lib.cfet_error_constant(self._ctx, C.c_void_p(psi0.data_ptr()), float(t0), float(T), int(n1),
                                                  int(order), self._sid(scheme), float(tol), float(ratio),
                                                  _stream_handle(stream), C.byref(c), C.byref(d), C.byref(h2)))
        return c.value, d.value, h2.value

    def select_dt(self, psi0, t0, T, target, T_probe, n_probe, order=4, tol=1e-10, scheme=None, ratio=2.0,
                  stream=None):
        """(dt, nsteps, c) for the accuracy goal `target` over a run of length T."""
        _check_vec(psi0, self.dim, "psi0")
        dt, n, c = C.c_double(), C.c_int64(), C.c_double()
        self._raise(self._lib.cfet_select_dt(self._ctx, C.c_void_p(psi0.data_ptr()), float(t0), float(T),
                                             float(target), float(T_probe), int(n_probe), int(order),
                                             self._sid(scheme), float(tol), float(ratio), _stream_handle(stream),
                                             C.byref(dt), C.byref(n), C.byref(c)))
        return dt.value, n.value, c.value

    def propagate_adaptive(self, psi, t0, T, target, h0, h_min, h_max, order=4, tol=1e-10, scheme=None,
                           max_steps=100000, forced_h=None, stream=None):
        """Adaptive CFET stepping of psi (in place) over [t0, t0 + T] for the
        goal `target` (cfet_propagate_adaptive);
        forced_h replays accepted steps.  Returns (accepted steps, trials, stats)."""
        _check_vec(psi, self.dim, "psi")
        cap = int(max_steps) if forced_h is None else len(forced_h)
        hlog = np.zeros(max(1, cap))
        fh = None if forced_h is None else np.ascontiguousarray(forced_h, dtype=np.float64)
        ns, nt = C.c_int64(), C.c_int64()
        st = _capi.cfet_stats()
        self._raise(self._lib.cfet_propagate_adaptive(
            self._ctx, C.c_void_p(psi.data_ptr()), float(t0), float(T), int(order), self._sid(scheme), float(tol),
            float(target), float(h0), float(h_min), float(h_max), int(max_steps),
            fh.ctypes.data_as(_capi.c_double_p) if fh is not None else None, 0 if fh is None else fh.size,
            hlog.ctypes.data_as(_capi.c_double_p), hlog.size, C.byref(ns), C.byref(nt), _stream_handle(stream),
            C.byref(st)))
        hs = list(fh) if fh is not None else hlog[: ns.value].tolist()
        return hs, nt.value, st.as_dict()

    def sync(self, stream=None):
        stats = _capi.cfet_stats()
        self._raise(self._lib.cfet_sync(self._ctx, _stream_handle(stream), C.byref(stats)))
        return stats.as_dict()


# ---------------------------------------------------------------- batches
@dataclass
class Chain:
    """One instance of a batch: the open XXZ chain (N, J, Delta, h) driven by
    f(t) sum_i a_i X_i with f a Python callable, or, when drive is None, the
    built-in A cos(omega t + phase) evaluated by the library."""
    N: int
    J: float
    Delta: float
    h: np.ndarray
    a: np.ndarray
    drive: object = None
    A: float = 0.0
    omega: float = 0.0
    phase: float = 0.0


def _decisions(nexp, log, keep):
    nsub = np.array([len(x) for x in log], dtype=np.int32)
    ks = np.array([k for x in log for k, _ in x], dtype=np.int32)
    hs = np.array([h for x in log for _, h in x], dtype=np.int32)
    keep += [nsub, ks, hs]
    return _capi.cfet_decisions(nexp, nsub.ctypes.data_as(_capi.c_int32_p), ks.ctypes.data_as(_capi.c_int32_p),
                                hs.ctypes.data_as(_capi.c_int32_p), len(ks), len(ks))


class BatchPropagator:
    """Many driven XXZ chains of uneven size propagated in one persistent launch
    (thread-block clusters for the large instances, a measured plan)."""

    def __init__(self, chains, *, m_max=16, m_min=2, max_substeps=64, precision="f64"):
        lib = _capi.load()
        self._keep = []
        arr = (_capi.cfet_chain * len(chains))()
        self._cbs = []
        self.dims = []
        for i, c in enumerate(chains):
            h = np.ascontiguousarray(c.h, dtype=np.float64)
            a = np.ascontiguousarray(c.a, dtype=np.float64)
            self._keep += [h, a]
            s = arr[i]
            s.nsites, s.J, s.Delta = c.N, c.J, c.Delta
            s.h = h.ctypes.data_as(_capi.c_double_p)
            s.a = a.ctypes.data_as(_capi.c_double_p)
            if c.drive is not None:
                cb = _capi.DRIVE_FN(lambda t, u, fn=c.drive: float(fn(t)))
                self._cbs.append(cb)
                s.f = cb
            s.A, s.omega, s.phase = c.A, c.omega, c.phase
            self.dims.append(1 << c.N)
        self._arr = arr
        opt = _capi.cfet_options()
        lib.cfet_options_default(C.byref(opt))
        opt.m_max, opt.m_min, opt.max_substeps = m_max, m_min, max_substeps
        opt.precision = _capi.PRECISIONS[precision]
        b = C.c_void_p()
        st = lib.cfet_batch_create(C.byref(b), len(chains), arr, C.byref(opt))
        if st != 0:
            raise CfetError(st, lib.cfet_batch_last_error(None).decode())
        self._lib, self._b, self.n = lib, b, len(chains)
        self.max_substeps = max_substeps

    def close(self):
        if getattr(self, "_b", None):
            self._lib.cfet_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, st):
        if st != 0:
            raise CfetError(st, self._lib.cfet_batch_last_error(self._b).decode())

    @property
    def plan(self):
        p = _capi.cfet_batch_plan()
        self._raise(self._lib.cfet_batch_get_plan(self._b, C.byref(p)))
        return {"cluster_size": p.cluster_size, "threads": p.threads, "coop_min_sites": p.coop_min_sites,
                "tuned_ms": p.tuned_ms}

    def set_plan(self, cluster_size, threads, coop_min_sites):
        p = _capi.cfet_batch_plan(cluster_size, threads, coop_min_sites, 0.0)
        self._raise(self._lib.cfet_batch_set_plan(self._b, C.byref(p)))

    def tune(self, t0, dt, order=6, tol=1e-10, nsteps=1, stream=None):
        p = _capi.cfet_batch_plan()
        self._raise(self._lib.cfet_batch_tune(self._b, float(t0), float(dt), int(order), float(tol), int(nsteps),
                                              _stream_handle(stream), C.byref(p)))
        return self.plan

    def propagate(self, psis, t0, dt, nsteps, order=6, tol=1e-10, stream=None, forced=None, record=False):
        """psis: list of CUDA complex128 tensors (one per instance), updated in
        place.  forced: per-instance decision logs to replay; record: also
        return the per-instance logs.  Returns per-instance stats."""
        if len(psis) != self.n:
            raise ValueError(f"expected {self.n} states")
        for t, d in zip(psis, self.dims):
            _check_vec(t, d, "psi")
        ptrs = (C.c_void_p * self.n)(*[t.data_ptr() for t in psis])
        s = {2: 1, 4: 2, 6: 5, 8: 11}.get(order, 1)
        nexp = int(nsteps) * s
        keep = []
        fd = None
        if forced is not None:
            fd = (_capi.cfet_decisions * self.n)(*[_decisions(nexp, lg, keep) for lg in forced])
        rd = None
        if record:
            rd = (_capi.cfet_decisions * self.n)()
            bufs = []
            for i in range(self.n):
                cap = max(1, nexp * self.max_substeps)
                rn, rk, rh = (np.zeros(nexp, np.int32), np.zeros(cap, np.int32), np.zeros(cap, np.int32))
                bufs.append((rn, rk, rh))
                rd[i] = _capi.cfet_decisions(nexp, rn.ctypes.data_as(_capi.c_int32_p),
                                             rk.ctypes.data_as(_capi.c_int32_p), rh.ctypes.data_as(_capi.c_int32_p),
                                             cap, 0)
        stats = (_capi.cfet_stats * self.n)()
        st = self._lib.cfet_batch_propagate(self._b, ptrs, float(t0), float(dt), int(nsteps), int(order), float(tol),
                                            _stream_handle(stream), fd, rd, stats)
        self._raise(st)
        out = [stats[i].as_dict() for i in range(self.n)]
        if record:
            logs = []
            for i, (rn, rk, rh) in enumerate(bufs):
                lg, pos = [], 0
                for e in range(nexp):
                    m = int(rn[e])
                    lg.append([(int(rk[pos + q]), int(rh[pos + q])) for q in range(m)])
                    pos += m
                logs.append(lg)
            return out, logs
        return out

    def kernel_time_ms(self):
        ms = C.c_float()
        self._raise(self._lib.cfet_batch_kernel_time_ms(self._b, C.byref(ms)))
        return float(ms.value)


def fidelity_loss(prop, amps, psi0, phi, t0, dt, nsteps, omega, phase=0.0, order=4, tol=1e-10,
                  checkpoint_every=None):
    """Differentiable L(amps) = 1 - |<phi|psi(T)>|^2 (torch scalar, float64):
    the forward call runs cfet_fidelity_grad once and keeps the gradient for
    the backward call."""
    import torch

    class _Fidelity(torch.autograd.Function):
        @staticmethod
        def forward(ctx, a):
            loss, grad, _ = prop.fidelity_grad(psi0, phi, t0, dt, nsteps, a.detach().cpu().numpy(), omega, phase,
                                               order, tol, checkpoint_every)
            ctx.save_for_backward(torch.from_numpy(grad).to(a.device, a.dtype))
            return torch.tensor(loss, dtype=a.dtype, device=a.device)

        @staticmethod
        def backward(ctx, g):
            (grad,) = ctx.saved_tensors
            return g * grad

    return _Fidelity.apply(amps)


def build():
    from .build import build as _b
    return _b()


__all__ = ["Propagator", "BatchPropagator", "Chain", "fidelity_loss", "XXZChain", "XField", "DIA", "PauliSum",
           "scheme_info", "CfetError",
           "SCHEME_IDS", "build"]
