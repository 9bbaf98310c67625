"""Host-side checks of the C-ABI library (no GPU compute calls).

The library must load, export every entry point declared in include/cfet.h,
reproduce the oracle's scheme tables in its host code, and reject invalid
arguments before touching a device.
"""

import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import schemes as S
import paper_1102_5071_gb300 as P
from paper_1102_5071_gb300 import _capi
from paper_1102_5071_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return _capi.load()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "cfet.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cfet_[a-z0-9_]+)\s*\(", text)) - {"cfet_drive_fn"})


def test_library_exports_every_declared_symbol(lib):
    syms = _declared_symbols()
    assert len(syms) >= 10
    for name in syms:
        assert hasattr(lib, name), name
    assert set(syms) == set(_capi.EXPORTED)


@pytest.mark.parametrize("name", list(S.SCHEMES))
def test_scheme_tables_match_oracle(lib, name):
    order, s, M, f, x, w, g = P.scheme_info(name)
    sc = S.SCHEMES[name]
    g_o, x_o, w_o, f_o = S.g_coefficients(sc)
    assert (order, s, M) == (sc.order, sc.s, sc.nA)
    assert np.max(np.abs(f - f_o)) < 1e-15
    assert np.max(np.abs(x - x_o)) < 1e-15 and np.max(np.abs(w - w_o)) < 1e-15
    assert np.max(np.abs(g - g_o)) < 1e-15


def test_scheme_info_rejects_unknown_id(lib):
    o = C.c_int32()
    assert lib.cfet_scheme_info(99, C.byref(o), None, None, None, None, None, None, 0) == _capi.CFET_EINVAL
    assert lib.cfet_scheme_info(0, C.byref(o), None, None, None, None, None, None, 0) == _capi.CFET_EINVAL


def _create(lib, h0, vs, fns, opt=None):
    ctx = C.c_void_p()
    varr = (_capi.cfet_op * max(1, len(vs)))(*vs)
    farr = (_capi.DRIVE_FN * max(1, len(fns)))(*fns)
    st = lib.cfet_create(C.byref(ctx), C.byref(h0), len(vs), varr, farr, None, C.byref(opt) if opt else None)
    return st, ctx


def test_create_validates_arguments(lib):
    keep = []
    h = np.zeros(4)
    ok_h0 = P._op_struct(P.XXZChain(4, 1.0, 0.5, h), keep)
    xf = P._op_struct(P.XField(4, np.ones(4)), keep)
    cb = _capi.DRIVE_FN(lambda t, u: 0.0)
    # mismatched chain length
    bad_v = P._op_struct(P.XField(5, np.ones(5)), keep)
    st, _ = _create(lib, ok_h0, [bad_v], [cb])
    assert st == _capi.CFET_EINVAL and b"X fields" in lib.cfet_last_error(None)
    # dim inconsistent with nsites
    bad = P._op_struct(P.XXZChain(4, 1.0, 0.5, h), keep)
    bad.dim = 17
    assert _create(lib, bad, [xf], [cb])[0] == _capi.CFET_EINVAL
    # non-finite field
    hn = np.array([0.0, np.nan, 0.0, 0.0])
    assert _create(lib, P._op_struct(P.XXZChain(4, 1.0, 0.5, hn), keep), [xf], [cb])[0] == _capi.CFET_EINVAL
    # options out of range
    opt = _capi.cfet_options()
    lib.cfet_options_default(C.byref(opt))
    opt.m_max = 65
    assert _create(lib, ok_h0, [xf], [cb], opt)[0] == _capi.CFET_EINVAL
    opt.m_max, opt.block_size = 16, 48
    assert _create(lib, ok_h0, [xf], [cb], opt)[0] == _capi.CFET_EINVAL
    # control-warp kernels (fixed point, complex64) take at most 2 x 384 + 32 threads
    for prec in (_capi.CFET_PREC_FX, _capi.CFET_PREC_C64):
        opt.block_size, opt.precision = 416, prec
        assert _create(lib, ok_h0, [xf], [cb], opt)[0] == _capi.CFET_EINVAL
    opt.block_size, opt.precision = 0, 7
    st, _ = _create(lib, ok_h0, [xf], [cb], opt)
    assert st == _capi.CFET_EINVAL and b"precision" in lib.cfet_last_error(None)
    opt.precision = _capi.CFET_PREC_DEFAULT
    # expansion method: known values only; Chebyshev is fixed point only
    opt.expm = 5
    st, _ = _create(lib, ok_h0, [xf], [cb], opt)
    assert st == _capi.CFET_EINVAL and b"expm" in lib.cfet_last_error(None)
    opt.expm, opt.precision = _capi.CFET_EXPM_CHEBYSHEV, _capi.CFET_PREC_C64
    st, _ = _create(lib, ok_h0, [xf], [cb], opt)
    assert st == _capi.CFET_EINVAL and b"CHEBYSHEV" in lib.cfet_last_error(None)
    opt.expm, opt.precision = _capi.CFET_EXPM_KRYLOV, _capi.CFET_PREC_DEFAULT
    # picture: known values; the interaction picture needs FP64, Krylov, a chain
    opt.picture = 3
    st, _ = _create(lib, ok_h0, [xf], [cb], opt)
    assert st == _capi.CFET_EINVAL and b"picture" in lib.cfet_last_error(None)
    opt.picture = _capi.CFET_PICTURE_INTERACTION    # with the default fixed-point precision
    st, _ = _create(lib, ok_h0, [xf], [cb], opt)
    assert st == _capi.CFET_EINVAL and b"INTERACTION" in lib.cfet_last_error(None)
    opt.precision = _capi.CFET_PREC_F64
    dia_ip = P._op_struct(P.DIA(np.array([0]), np.ones((1, 8))), keep)
    st, _ = _create(lib, dia_ip, [], [], opt)
    assert st == _capi.CFET_EINVAL and b"INTERACTION" in lib.cfet_last_error(None)
    opt.picture, opt.precision = _capi.CFET_PICTURE_SCHROEDINGER, _capi.CFET_PREC_DEFAULT
    # re-orthogonalisation: 0 or 1, FP64 Krylov only
    opt.reorth = 2
    st, _ = _create(lib, ok_h0, [xf], [cb], opt)
    assert st == _capi.CFET_EINVAL and b"reorth" in lib.cfet_last_error(None)
    opt.reorth = 1                                    # with the default fixed-point precision
    st, _ = _create(lib, ok_h0, [xf], [cb], opt)
    assert st == _capi.CFET_EINVAL and b"reorth" in lib.cfet_last_error(None)
    opt.reorth = 0
    # DIA offsets out of range
    dia = P._op_struct(P.DIA(np.array([0, 7]), np.ones((2, 7))), keep)
    assert _create(lib, dia, [], [])[0] == _capi.CFET_EINVAL


def test_create_validates_pauli_sums(lib):
    # CFET_OP_PAULI: FP64 only, masks below nsites, finite coefficients, at most
    # 4096 strings, only with chains and X fields, no interaction picture; all
    # checked before any device work
    keep = []
    cb = _capi.DRIVE_FN(lambda t, u: 0.0)
    ps = P._op_struct(P.PauliSum(4, [(0.5, "XYZI"), (-0.3, "IIZZ")]), keep)
    xf = P._op_struct(P.XField(4, np.ones(4)), keep)
    opt = _capi.cfet_options()
    lib.cfet_options_default(C.byref(opt))
    for prec in (_capi.CFET_PREC_FX, _capi.CFET_PREC_C64):
        opt.precision = prec
        st, _ = _create(lib, ps, [xf], [cb], opt)
        assert st == _capi.CFET_EINVAL and b"CFET_PREC_F64" in lib.cfet_last_error(None)
    opt.precision = _capi.CFET_PREC_DEFAULT
    opt.expm = _capi.CFET_EXPM_CHEBYSHEV            # the default precision of a Pauli sum is FP64
    st, _ = _create(lib, ps, [xf], [cb], opt)
    assert st == _capi.CFET_EINVAL and b"CHEBYSHEV" in lib.cfet_last_error(None)
    opt.expm, opt.precision, opt.picture = _capi.CFET_EXPM_KRYLOV, _capi.CFET_PREC_F64, _capi.CFET_PICTURE_INTERACTION
    chain = P._op_struct(P.XXZChain(4, 1.0, 0.5, np.zeros(4)), keep)
    st, _ = _create(lib, chain, [ps], [cb], opt)       # a Pauli drive makes it a Pauli-sum context
    assert st == _capi.CFET_EINVAL and b"INTERACTION" in lib.cfet_last_error(None)
    bad = P._op_struct(P.PauliSum(4, [(0.5, "XYZI")]), keep)
    bad.xmask[0] = 1 << 4                              # beyond the chain
    st, _ = _create(lib, bad, [], [])
    assert st == _capi.CFET_EINVAL and b"mask" in lib.cfet_last_error(None)
    nan = P._op_struct(P.PauliSum(4, [(float("nan"), "XIII")]), keep)
    assert _create(lib, nan, [], [])[0] == _capi.CFET_EINVAL
    big = P._op_struct(P.PauliSum(4, [(0.1, "ZIII")] * 4097), keep)
    st, _ = _create(lib, big, [], [])
    assert st == _capi.CFET_EINVAL and b"4096" in lib.cfet_last_error(None)
    other = P._op_struct(P.PauliSum(5, [(0.5, "XIIII")]), keep)   # another chain length
    assert _create(lib, ps, [other], [cb])[0] == _capi.CFET_EINVAL
    dia = P._op_struct(P.DIA(np.array([0]), np.ones((1, 16))), keep)
    st, _ = _create(lib, ps, [dia], [cb])
    assert st == _capi.CFET_EINVAL and b"Pauli" in lib.cfet_last_error(None)


def test_pauli_labels_give_masks():
    ps = P.PauliSum(5, [(0.5, "XYZII"), (1.5, {4: "Y", 1: "z"}), (-2.0, "IIIII")])
    assert list(ps.xmask) == [0b00011, 0b10000, 0] and list(ps.zmask) == [0b00110, 0b10010, 0]
    assert list(ps.coeff) == [0.5, 1.5, -2.0]
    with pytest.raises(ValueError):
        P.PauliSum(3, [(1.0, {3: "X"})])
    with pytest.raises(ValueError):
        P.PauliSum(3, [(1.0, "XQZ")])


@pytest.mark.parametrize("tile_bits,nsites,windows", [(11, 13, 2), (11, 19, 3), (11, 26, 4),
                                                      (12, 13, 2), (12, 20, 3), (12, 27, 4)])
def test_window_tiling_of_long_chains(lib, tile_bits, nsites, windows):
    # the index arithmetic of the tiled apply (fixed point: tiles of 2^11,
    # complex64: 2^12), run on the host from the kernels' own header: every
    # index once per window, every flip and bond in one window, copy units
    # contiguous; `windows` passes visit windows * 2^nsites indices
    n = C.c_int64()
    assert lib.cfet_selftest_tiling(nsites, tile_bits, C.byref(n)) == _capi.CFET_OK, lib.cfet_last_error(None)
    assert n.value == windows << nsites


@pytest.mark.parametrize("tile_bits", [11, 12])
def test_window_tiling_every_chain_length(lib, tile_bits):
    # every chain length the tiled kernels can take up to 24 sites: the window
    # cover and, for both kernels, every TMA box slot of every tile of three
    # basis vectors against the tiling (the maps are built the same way at
    # run time, so a geometry that fails here never reaches the GPU)
    for nsites in range(max(tile_bits, 13), 25):
        n = C.c_int64()
        assert lib.cfet_selftest_tiling(nsites, tile_bits, C.byref(n)) == _capi.CFET_OK, (nsites, lib.cfet_last_error(None))
        assert n.value >= 2 << nsites


def test_window_tiling_selftest_validates(lib):
    n = C.c_int64()
    assert lib.cfet_selftest_tiling(20, 10, C.byref(n)) == _capi.CFET_EINVAL
    assert lib.cfet_selftest_tiling(10, 11, C.byref(n)) == _capi.CFET_EINVAL
    assert lib.cfet_selftest_tiling(28, 12, C.byref(n)) == _capi.CFET_EINVAL
    assert lib.cfet_selftest_tiling(20, 12, None) == _capi.CFET_EINVAL


def test_options_default(lib):
    opt = _capi.cfet_options()
    lib.cfet_options_default(C.byref(opt))
    assert (opt.m_max, opt.m_min, opt.max_substeps, opt.block_size) == (16, 2, 64, 0)
    assert opt.barrier_timeout_s == 2.0
    assert opt.expm == _capi.CFET_EXPM_KRYLOV and opt.picture == _capi.CFET_PICTURE_SCHROEDINGER
    assert opt.precision == _capi.CFET_PREC_DEFAULT and opt.reorth == 0


def test_no_device_gives_enodev(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    keep = []
    h0 = P._op_struct(P.XXZChain(3, 1.0, 0.5, np.zeros(3)), keep)
    st, ctx = _create(lib, h0, [], [])
    assert st == _capi.CFET_ENODEV and not ctx.value


def test_binding_refuses_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(_capi, "_lib", None)
    monkeypatch.setattr(_capi, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _capi.load()


def _chain_arr(specs, keep):
    arr = (_capi.cfet_chain * len(specs))()
    for i, (N, h, a) in enumerate(specs):
        h = np.ascontiguousarray(h, dtype=np.float64)
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep += [h, a]
        arr[i].nsites, arr[i].J, arr[i].Delta = N, 1.0, 0.5
        arr[i].h = h.ctypes.data_as(_capi.c_double_p) if h.size else None
        arr[i].a = a.ctypes.data_as(_capi.c_double_p)
        arr[i].A, arr[i].omega = 1.0, 2.0
    return arr


def test_batch_create_validates_arguments(lib):
    keep = []
    b = C.c_void_p()
    ok = _chain_arr([(4, np.zeros(4), np.ones(4))], keep)
    assert lib.cfet_batch_create(C.byref(b), 0, ok, None) == _capi.CFET_EINVAL
    big = _chain_arr([(25, np.zeros(25), np.ones(25))], keep)
    assert lib.cfet_batch_create(C.byref(b), 1, big, None) == _capi.CFET_EINVAL
    assert b"nsites" in lib.cfet_batch_last_error(None)
    nan = _chain_arr([(3, np.array([0.0, np.nan, 0.0]), np.ones(3))], keep)
    assert lib.cfet_batch_create(C.byref(b), 1, nan, None) == _capi.CFET_EINVAL
    nul = _chain_arr([(3, np.zeros(0), np.ones(3))], keep)
    assert lib.cfet_batch_create(C.byref(b), 1, nul, None) == _capi.CFET_EINVAL
    opt = _capi.cfet_options()
    lib.cfet_options_default(C.byref(opt))
    opt.precision = _capi.CFET_PREC_FX      # batches run FP64 or complex64
    assert lib.cfet_batch_create(C.byref(b), 1, ok, C.byref(opt)) == _capi.CFET_EINVAL
    assert not b.value


def test_batch_no_device_gives_enodev(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    keep = []
    b = C.c_void_p()
    ok = _chain_arr([(4, np.zeros(4), np.ones(4)), (6, np.zeros(6), np.ones(6))], keep)
    assert lib.cfet_batch_create(C.byref(b), 2, ok, None) == _capi.CFET_ENODEV and not b.value


def test_wait_selftest_validates(lib):
    st = C.c_int32(0)
    assert lib.cfet_selftest_wait_timeout(2, 0.1, C.byref(st)) == _capi.CFET_EINVAL
    assert lib.cfet_selftest_wait_timeout(0, 0.0, C.byref(st)) == _capi.CFET_EINVAL
    assert lib.cfet_selftest_wait_timeout(0, 20.0, C.byref(st)) == _capi.CFET_EINVAL
    assert lib.cfet_selftest_wait_timeout(0, 0.1, None) == _capi.CFET_EINVAL


# ---------------------------------------------------------------- Chebyshev coefficients (host only)
@pytest.mark.parametrize("z", [1e-3, 0.5, 3.0, -7.3, 40.0, 300.0])
@pytest.mark.parametrize("tol", [1e-6, 1e-10, 0.0])
def test_chebyshev_coefficients_match_library_bessel(lib, z, tol):
    # r_k = (2 - delta_k0) J_k(z) from Miller's recurrence against scipy's J_k,
    # and the same truncation order as the oracle's rule
    from scipy import special
    from oracle import chebyshev as CH
    r, K, tail = P.chebyshev_coefficients(z, tol)
    ref = special.jv(np.arange(K + 1), z)
    ref[1:] *= 2.0
    assert np.max(np.abs(r - ref)) <= 1e-14 * max(1.0, abs(z)) ** 0.5
    r_o, K_o, tail_o = CH.coefficients(z, tol)
    assert K == K_o and abs(tail - tail_o) <= 1e-14
    assert tail <= (tol if tol > 0 else 2.0 ** -52)


def test_chebyshev_coefficients_closed_forms(lib):
    # z = 0: exp(0) = T_0 only; the normalisation J_0 + 2 sum J_2k = 1 and
    # sum_k r_k (-i)^k T_k(1) = exp(-i z) (Jacobi-Anger at x = 1)
    r, K, tail = P.chebyshev_coefficients(0.0, 1e-12)
    assert K == 0 and r.tolist() == [1.0] and tail == 0.0
    for z in (0.9, 12.0, 150.0):
        r, K, _ = P.chebyshev_coefficients(z, 0.0)
        assert abs(r[0] + r[2::2].sum() - 1.0) <= 1e-14
        s = sum(r[k] * (-1j) ** k for k in range(K + 1))
        assert abs(s - np.exp(-1j * z)) <= 1e-13


def test_chebyshev_coefficients_validate(lib):
    K, tail = C.c_int32(), C.c_double()
    assert lib.cfet_chebyshev_coefficients(float("nan"), 1e-8, 0, None, C.byref(K), C.byref(tail)) == _capi.CFET_EINVAL
    assert lib.cfet_chebyshev_coefficients(2e8, 1e-8, 0, None, C.byref(K), C.byref(tail)) == _capi.CFET_EINVAL
    buf = np.zeros(2)
    st = lib.cfet_chebyshev_coefficients(10.0, 1e-8, 2, buf.ctypes.data_as(_capi.c_double_p), C.byref(K), C.byref(tail))
    assert st == _capi.CFET_EINVAL and K.value > 1


def test_create_validates_csr_operators(lib):
    # CFET_OP_CSR: structure, column range, finite values and Hermiticity are
    # checked before any device work; a valid operator then reaches the device
    # check (CFET_ENODEV without a GPU)
    keep = []
    cb = _capi.DRIVE_FN(lambda t, u: 0.0)
    rp = np.array([0, 1, 2], dtype=np.int64)
    herm = P.CSR(rp, np.array([1, 0]), np.array([0.5 + 0.25j, 0.5 - 0.25j]))
    cases = [
        (P.CSR(rp, np.array([1, 0]), np.array([0.5 + 0.25j, 0.5 + 0.25j])), b"Hermitian"),
        (P.CSR(rp, np.array([2, 0]), np.array([1.0, 1.0])), b"column"),
        (P.CSR(np.array([0, 2, 1], dtype=np.int64), np.array([0, 1]), np.array([1.0, 1.0])), b"row_ptr"),
        (P.CSR(np.array([1, 1, 2], dtype=np.int64), np.array([0, 1]), np.array([1.0, 1.0])), b"row_ptr"),
        (P.CSR(np.array([0, 1], dtype=np.int64), np.array([0]), np.array([1.0 + 0.5j])), b"Hermitian"),
        (P.CSR(rp, np.array([1, 0]), np.array([np.inf, np.inf])), b"finite"),
    ]
    for op, word in cases:
        st, _ = _create(lib, P._op_struct(op, keep), [], [])
        assert st == _capi.CFET_EINVAL and word in lib.cfet_last_error(None), (word, lib.cfet_last_error(None))
    # drive operators of a CSR H0 must be CSR of the same dimension
    dia = P._op_struct(P.DIA(np.array([0]), np.ones((1, 2))), keep)
    st, _ = _create(lib, P._op_struct(herm, keep), [dia], [cb])
    assert st == _capi.CFET_EINVAL and b"CSR" in lib.cfet_last_error(None)
    other = P.CSR(np.array([0, 1, 2, 3], dtype=np.int64), np.array([0, 1, 2]), np.ones(3))
    st, _ = _create(lib, P._op_struct(herm, keep), [P._op_struct(other, keep)], [cb])
    assert st == _capi.CFET_EINVAL
    # mirrors within the tolerance, duplicates summed, empty rows: valid
    dup = P.CSR(np.array([0, 3, 4, 4], dtype=np.int64), np.array([1, 0, 1, 0]),
                np.array([0.25 + 0.5j, 2.0, 0.25 + 0.5j, 0.5 - 1.0j]))
    for op in (herm, dup):
        st, ctx = _create(lib, P._op_struct(op, keep), [], [])
        assert st in (_capi.CFET_OK, _capi.CFET_ENODEV), lib.cfet_last_error(None)
        if st == _capi.CFET_OK:
            lib.cfet_destroy(ctx)
