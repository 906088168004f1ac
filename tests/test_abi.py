"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/dg.h declares, and its host-only helpers (reference
basis and quadrature) are right."""
import math

import numpy as np
import pytest

from paper_1502_02941_gb300 import dg as D


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    return D.load()


def test_exports_every_declared_symbol(lib):
    syms = D.header_symbols()
    assert len(syms) >= 20
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing
    # the binding wraps every declared entry point under the same name
    assert set(syms) <= set(D._SIGS)
    for s in syms:
        assert callable(getattr(D, s))


def test_status_strings(lib):
    for code in range(10):
        assert D.dg_status_string(code).startswith("DG_")
    assert "unknown" in D.dg_status_string(99)


def test_params_default(lib):
    p = D.dg_params_default()
    assert (p.method, p.degree, p.gmres_m, p.max_it, p.precond) == (D.DG_SIPG, 1, 50, 10000, 1)
    assert p.sigma_bdry_factor == 2.0 and p.b0 == 1.0 and p.tol == 1e-10


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(D.DGError):
        D.dg_create(0)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_reference_basis_orthonormal(lib, k):
    """int_T phi_i phi_j = delta_ij on the reference triangle (area 1/2), with the
    library's own volume rule, which is exact for degree 2k."""
    rs, w = D.dg_reference_rule(D.DG_POINTS_VOLUME, k)
    assert abs(w.sum() - 0.5) < 1e-15 and len(w) == (k + 2) ** 2
    phi, _, _ = D.dg_reference_basis(k, rs)
    M = phi.T @ (w[:, None] * phi)
    np.testing.assert_allclose(M, np.eye(phi.shape[1]), atol=1e-13)
    # spans P_k: monomials r^a s^b are reproduced by projection
    for a in range(k + 1):
        for b in range(k + 1 - a):
            f = rs[:, 0] ** a * rs[:, 1] ** b
            c = phi.T @ (w * f)
            np.testing.assert_allclose(phi @ c, f, atol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_reference_basis_gradients(lib, k):
    rng = np.random.default_rng(k)
    r = rng.uniform(0.05, 0.6, 20)
    s = rng.uniform(0.05, 0.3, 20)
    rs = np.stack([r, s], 1)
    phi, dr, ds = D.dg_reference_basis(k, rs)
    h = 1e-6
    fr = (D.dg_reference_basis(k, rs + [h, 0])[0] - D.dg_reference_basis(k, rs - [h, 0])[0]) / (2 * h)
    fs = (D.dg_reference_basis(k, rs + [0, h])[0] - D.dg_reference_basis(k, rs - [0, h])[0]) / (2 * h)
    np.testing.assert_allclose(dr, fr, atol=1e-7)
    np.testing.assert_allclose(ds, fs, atol=1e-7)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_reference_rules(lib, k):
    t, w = D.dg_reference_rule(D.DG_POINTS_BOUNDARY, k)
    x, wx = np.polynomial.legendre.leggauss(k + 2)
    np.testing.assert_allclose(t[:, 0], 0.5 * (x + 1), atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * wx, atol=1e-15)
    # the L2-error rule integrates r^a s^b exactly to degree 2k+6
    rs, w = D.dg_reference_rule(D.DG_POINTS_ERROR, k)
    for a in range(2 * k + 7):
        for b in range(2 * k + 7 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs((w * rs[:, 0] ** a * rs[:, 1] ** b).sum() - exact) < 1e-15


def test_invalid_arguments(lib):
    with pytest.raises(D.DGError):
        D.dg_reference_basis(7, np.zeros((1, 2)))


def _declared_arity():
    """Parameter count of every entry point in include/dg.h (comments removed)."""
    import re
    txt = open(D.HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    txt = re.sub(r"//[^\n]*", "", txt)
    out = {}
    for m in re.finditer(r"(dg_status|const char\s*\*|size_t)\s+(dg_\w+)\s*\(([^)]*)\)\s*;", txt):
        args = m.group(3).strip()
        out[m.group(2)] = (m.group(1).replace(" ", ""), 0 if args in ("", "void") else args.count(",") + 1)
    return out


def test_binding_signatures_match_the_header(lib):
    """The binding passes exactly as many arguments as each declaration takes,
    and declares the same result kind (status int, string or size)."""
    import ctypes
    kinds = {"dg_status": ctypes.c_int, "constchar*": ctypes.c_char_p, "size_t": ctypes.c_size_t}
    arity = _declared_arity()
    assert set(arity) == set(D.header_symbols())
    for name, (ret, n) in arity.items():
        res, args = D._SIGS[name]
        assert len(args) == n, (name, len(args), n)
        assert res is kinds[ret], (name, res, ret)


def test_binding_refuses_host_tensors_for_device_arguments():
    """Every pointer argument is marked host or device in the binding.  Device
    arguments take CUDA tensors (or raw integer addresses); a numpy array or a
    CPU tensor there is refused before any library call, because the kernels
    would dereference its host address.  Host arguments take numpy arrays (or
    CPU tensors).  Sizes and dtypes are checked against what the call needs."""
    import torch
    with pytest.raises(ValueError):
        D._dev(torch.zeros(4, dtype=torch.float64))          # CPU tensor as device memory
    with pytest.raises(ValueError):
        D._dev(np.zeros(4))                                  # numpy array as device memory
    with pytest.raises(ValueError):
        D._host(np.zeros((4, 2))[:, 0])                      # not contiguous
    with pytest.raises(ValueError):
        D._host(np.zeros(3), n=4)                            # too few elements
    with pytest.raises(ValueError):
        D._host(np.zeros(3, np.float32), dtype="f64")        # wrong dtype
    a = np.zeros(3)
    assert D._host(a) == a.ctypes.data and D._host(None) is None and D._host(7) == 7
    assert D._dev(None) is None and D._dev(7) == 7
    t = torch.zeros(3, dtype=torch.float64)
    assert D._host(t) == t.data_ptr()
    # the wrappers refuse host memory for device arguments before calling the
    # library (no handle is needed for the refusal)
    for fn in (D.dg_l2_error_noalloc, D.dg_l2_error):
        with pytest.raises(ValueError):
            fn(None, np.zeros(3), np.zeros(3))
        with pytest.raises(ValueError):
            fn(None, torch.zeros(3, dtype=torch.float64), torch.zeros(3, dtype=torch.float64))
    with pytest.raises(ValueError):
        D.dg_apply(None, D.DG_F64, np.zeros(3), np.zeros(3))
    with pytest.raises(ValueError):
        D.dg_gmres_solve(None, None, np.zeros(3))


def test_network_checkpoint_round_trip():
    """Trained weights are saved with a header (degree, size, seed, settings)
    and read back bit for bit; foreign, truncated or mismatched files are
    refused (in memory: the format is the same for files)."""
    import io
    from paper_1502_02941_gb300 import learned as L
    n = D.dg_mlp_num_params(2)
    theta = np.random.default_rng(0).standard_normal(n).astype(np.float32)
    buf = io.BytesIO()
    L.save_weights(buf, theta, 2, seed=7, config={"steps": 4000})
    raw = buf.getvalue()
    back, head = L.load_weights(io.BytesIO(raw))
    np.testing.assert_array_equal(back, theta)
    assert head["degree"] == 2 and head["seed"] == 7 and head["config"] == {"steps": 4000}
    assert raw[:8] == b"DGMLPW1\0" and len(raw) == 12 + int.from_bytes(raw[8:12], "little") + 4 * n
    with pytest.raises(ValueError):
        L.save_weights(io.BytesIO(), theta[:-1], 2)
    for bad in (b"X" + raw[1:], raw[:-4]):
        with pytest.raises(ValueError):
            L.load_weights(io.BytesIO(bad))
    # headers that are not an object with an integer degree in 1..3 are refused
    # with ValueError too (not KeyError / AttributeError / DGError)
    import json
    import struct
    for h in ({"n_params": n, "dtype": "float32"}, {"degree": 7, "n_params": n, "dtype": "float32"},
              {"degree": "2", "n_params": n, "dtype": "float32"}, [2, n], "x"):
        hb = json.dumps(h).encode()
        blob = raw[:8] + struct.pack("<I", len(hb)) + hb + theta.tobytes()
        with pytest.raises(ValueError):
            L.load_weights(io.BytesIO(blob))
    hb = b"\xff\xfe{"
    with pytest.raises(ValueError):
        L.load_weights(io.BytesIO(raw[:8] + struct.pack("<I", len(hb)) + hb))
