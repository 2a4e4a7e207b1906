"""The C ABI library loads, exports every entry point include/pp.h declares,
and its host-only logic (argument validation, Eq. "l2cost" coefficients)
behaves as documented.  No device work is issued here."""
import ctypes
import os
import re
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2204_10252_gb300.build import build_library
    import paper_2204_10252_gb300 as pp
    build_library()
    return pp.lib()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(pp_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert len(names) >= 13
    for n in sorted(names):
        assert hasattr(L, n), "missing export %s" % n


def test_binding_covers_every_symbol():
    import paper_2204_10252_gb300.binding as b
    for n in declared_symbols():
        assert n in b._SIGS, "binding lacks %s" % n


def test_poly_coeffs_match_golden_rationals(L):
    import paper_2204_10252_gb300 as pp
    table = {}
    with open(os.path.join(ROOT, "tests", "golden", "l2_coeffs.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                d, rest = line.split(":")
                table[int(d)] = [float(Fraction(t)) for t in rest.split()]
    for d in range(0, 9):
        got = pp.pp_poly_coeffs_l2(d)
        ref = np.array(table[d])
        # exact integer ratios, rounded once to double
        assert np.max(np.abs(got - ref) / np.abs(ref)) <= 2e-16, d


def test_invalid_arguments_are_rejected_without_device_work(L):
    import paper_2204_10252_gb300 as pp
    from paper_2204_10252_gb300.binding import pp_dims, pp_sampling
    with pytest.raises(pp.PPError) as e:
        pp.pp_poly_coeffs_l2(9)
    assert e.value.status == 1
    out = ctypes.c_void_p(0)
    d = pp_dims()
    d.ndim = 2
    d.n[0] = d.n[1] = 64
    s = pp_sampling()
    assert L.pp_plan_create(None, d, 4, ctypes.c_void_p(16), ctypes.byref(s), 0, 0, None) == 1
    assert L.pp_plan_create(ctypes.byref(out), d, 4, None, ctypes.byref(s), 0, 0, None) == 1
    d.ndim = 4
    assert L.pp_plan_create(ctypes.byref(out), d, 4, ctypes.c_void_p(16), ctypes.byref(s), 0, 0, None) == 2
    assert "ndim" in pp.pp_last_error()
    d.ndim = 2
    assert L.pp_plan_create(ctypes.byref(out), d, 0, ctypes.c_void_p(16), ctypes.byref(s), 0, 0, None) == 1
    d.n[0] = 66
    assert L.pp_plan_create(ctypes.byref(out), d, 4, ctypes.c_void_p(16), ctypes.byref(s), 0, 0, None) == 2
    assert out.value is None
    # Toeplitz-embedded normal operator: coils <= 32 and 2n a register transform length
    traj = (ctypes.c_float * 2)(0.0, 0.0)
    st = pp_sampling()
    st.kind = 2
    st.traj = ctypes.cast(traj, ctypes.c_void_p)
    st.K = 1
    st.kb_width = 4
    st.oversamp = 1.25
    d.n[0] = d.n[1] = 80
    assert L.pp_plan_create(ctypes.byref(out), d, 4, ctypes.c_void_p(16), ctypes.byref(st), 0, 0, None) == 2
    assert "Toeplitz" in pp.pp_last_error()
    d.n[0] = d.n[1] = 64
    assert L.pp_plan_create(ctypes.byref(out), d, 33, ctypes.c_void_p(16), ctypes.byref(st), 0, 0, None) == 2
    assert out.value is None
    st.kind = 3
    assert L.pp_plan_create(ctypes.byref(out), d, 4, ctypes.c_void_p(16), ctypes.byref(st), 0, 0, None) == 1
    # prox: levels outside 1..2 and axes not multiples of 2^levels
    d.n[0] = 64
    assert L.pp_prox_l1_haar(d, 3, ctypes.c_float(0.1), ctypes.c_void_p(16), ctypes.c_void_p(16), None) == 2
    d.n[0] = 62
    assert L.pp_prox_l1_haar(d, 2, ctypes.c_float(0.1), ctypes.c_void_p(16), ctypes.c_void_p(16), None) == 2
    assert L.pp_prox_l1_haar(d, 1, ctypes.c_float(-1.0), ctypes.c_void_p(16), ctypes.c_void_p(16), None) == 1
    # Daubechies-4 prox: 2-D, levels 1..4, axes <= 512 and multiples of 2^levels
    d.n[0] = 64
    assert L.pp_prox_l1_db4(d, 5, ctypes.c_float(0.1), ctypes.c_void_p(16), ctypes.c_void_p(16), None) == 2
    d.n[0] = 40
    assert L.pp_prox_l1_db4(d, 4, ctypes.c_float(0.1), ctypes.c_void_p(16), ctypes.c_void_p(16), None) == 2
    d.n[0] = 1024
    assert L.pp_prox_l1_db4(d, 1, ctypes.c_float(0.1), ctypes.c_void_p(16), ctypes.c_void_p(16), None) == 2
    d.ndim = 3
    d.n[0] = d.n[2] = 16
    assert L.pp_prox_l1_db4(d, 1, ctypes.c_float(0.1), ctypes.c_void_p(16), ctypes.c_void_p(16), None) == 2
    d.ndim = 2
    d.n[0] = 64
    assert L.pp_prox_l1_db4(d, 2, ctypes.c_float(-0.5), ctypes.c_void_p(16), ctypes.c_void_p(16), None) == 1
    d.n[0] = 62
    # solve / applies with NULL plans
    assert L.pp_normal_apply(None, ctypes.c_void_p(16), ctypes.c_void_p(32), None) == 1
    assert L.pp_fista_solve(None, ctypes.c_void_p(16), ctypes.c_float(0.1), 1, None, 0,
                            ctypes.c_void_p(16), None, None) == 1
    assert L.pp_plan_destroy(None) == 0


def test_binding_rejects_wrong_sizes_before_device_work(L):
    # The C ABI sees raw pointers only; the binding compares element counts
    # with the plan's shapes and raises before calling into the library.
    import torch
    import paper_2204_10252_gb300 as pp
    from paper_2204_10252_gb300.binding import Batch, Plan
    with pytest.raises(ValueError):
        pp.pp_plan_create((32, 32), 2, torch.zeros(3 * 32 * 32, dtype=torch.complex64),
                          mask=np.ones((32, 32), np.uint8), power_iters=0)
    with pytest.raises(ValueError):
        pp.pp_plan_create((32, 32), 2, torch.zeros(2 * 32 * 32, dtype=torch.complex64),
                          mask=np.ones((16, 32), np.uint8), power_iters=0)
    fake = Plan(0, (32, 32), 2, None, (2, 32, 32))
    x = torch.zeros(32 * 32, dtype=torch.complex64)
    with pytest.raises(ValueError):
        pp.pp_normal_apply(fake, x, torch.zeros(32 * 31, dtype=torch.complex64))
    with pytest.raises(ValueError):
        pp.pp_adjoint_apply(fake, torch.zeros(32 * 32, dtype=torch.complex64), x)
    with pytest.raises(ValueError):
        pp.pp_adjoint_apply_static(fake, torch.zeros(2 * 32 * 33, dtype=torch.complex64), x)
    with pytest.raises(ValueError):
        pp.pp_fista_solve(fake, torch.zeros(2 * 32 * 32 + 1, dtype=torch.complex64), 0.1, 1,
                          None, 0, x)
    with pytest.raises(ValueError):
        pp.pp_prox_l1_haar((32, 32), 2, 0.1, x, torch.zeros(10, dtype=torch.complex64))
    fb = Batch(0, [(8, 8), (4, 8)], [1, 2], [], np.array([0, 64, 96]), np.array([0, 64, 128]))
    with pytest.raises(ValueError):
        pp.pp_batch_normal_apply(fb, torch.zeros(95, dtype=torch.complex64),
                                 torch.zeros(96, dtype=torch.complex64))
    fake.handle = None
    fb.handle = None


@pytest.mark.parametrize("d,mu", [(0, 0.2), (1, 0.1), (3, 0.05), (5, 0.02), (8, 0.3)])
def test_chebyshev_coefficients_match_oracle(L, d, mu):
    import paper_2204_10252_gb300 as pp
    from oracle import pp_oracle as O
    got = pp.pp_poly_coeffs_cheb(d, mu)
    ref = np.array(O.poly_coeffs_cheb(d, mu))
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    with pytest.raises(pp.PPError):
        pp.pp_poly_coeffs_cheb(3, 1.5)


@pytest.mark.parametrize("kind,d,mu", [("l2", 0, 0), ("l2", 3, 0), ("l2", 5, 0), ("cheb", 5, 1e-3),
                                        ("cheb", 3, 0.2), ("cheb", 8, 0.05)])
def test_poly_max_zp_matches_oracle(L, kind, d, mu):
    # host-only entry point: max over [0, 1] of z p(z) against the oracle's
    # dense grid, and 1 + 1/T_{d+1}(a) for the Chebyshev design
    import math
    import paper_2204_10252_gb300 as pp
    from oracle import pp_oracle as O
    c = [float(v) for v in (O.poly_coeffs_l2(d) if kind == "l2" else O.poly_coeffs_cheb(d, mu))]
    got = pp.pp_poly_max_zp(c, d)
    assert abs(got - O.poly_max_zp(c)) <= 1e-8 * got
    if kind == "cheb":
        a = (1 + mu) / (1 - mu)
        assert abs(got - (1 + 1 / math.cosh((d + 1) * math.acosh(a)))) <= 1e-8


@pytest.mark.parametrize("d", [0, 1, 3, 5, 8])
@pytest.mark.parametrize("terms", [[(1, 0)], [(1, 1)], [(1, 0), (3, 2)], [(2, 0), (-1, 1)], [(1, 6)]])
def test_weighted_l2_coefficients_match_oracle(L, d, terms):
    # host-only entry point: the library's LU + refinement against the
    # oracle's exact rational solution of Eq. "wl2cost"
    import paper_2204_10252_gb300 as pp
    from oracle import pp_oracle as O
    # the normal equations are Hankel (Hilbert-like: condition ~1e13 at d = 8),
    # so rounding the moments to double already moves the solution by up to
    # cond * 1e-16; the oracle therefore solves, exactly, the system of the
    # same double moments the library receives
    mom = [float(sum(Fraction(a) / (k + e + 1) for a, e in terms)) for k in range(2 * d + 3)]
    ref = np.array([float(v) for v in O.poly_coeffs_wl2(d, [Fraction(m) for m in mom])])
    got = pp.pp_poly_coeffs_wl2(d, mom)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    if terms == [(1, 0)] and d <= 3:
        assert np.max(np.abs(got - pp.pp_poly_coeffs_l2(d))) <= 1e-10 * np.max(np.abs(ref))


def test_weighted_l2_rejects_a_zero_weight(L):
    import paper_2204_10252_gb300 as pp
    with pytest.raises(pp.PPError) as e:
        pp.pp_poly_coeffs_wl2(3, np.zeros(9))
    assert e.value.status == 1
    with pytest.raises(ValueError):
        pp.pp_poly_coeffs_wl2(3, np.ones(5))


def test_binding_structs_match_the_header_layout(tmp_path):
    # the ctypes structures of the binding against the C compiler's layout of
    # the same structs in include/pp.h (sizes and field offsets)
    import shutil
    import subprocess
    from paper_2204_10252_gb300 import binding as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    checks = {"pp_dims": ["ndim", "n"], "pp_sampling": ["kind", "mask", "traj", "K", "kb_width", "oversamp"],
              "pp_solve_info": ["rescale", "levels", "no_momentum", "history", "ref", "bnorm", "L",
                                "launches", "wavelet", "safe_scale"]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pp.h"', "int main(void) {"]
    for st, fields in checks.items():
        lines.append('    printf("%%zu\\n", sizeof(%s));' % st)
        for f in fields:
            lines.append('    printf("%%zu\\n", offsetof(%s, %s));' % (st, f))
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for st, fields in checks.items():
        cls = getattr(B, st)
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f).offset for f in fields]
    assert got == want


def test_readme_example_uses_the_binding_as_declared():
    # every pp.* call in the README's Python example names a function of the
    # package, and its keyword arguments are parameters of that function
    import inspect
    import paper_2204_10252_gb300 as pkg
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "README.md")).read()
    code = re.search(r"```python\n(.*?)```", text, re.S).group(1)
    calls = re.findall(r"pp\.(\w+)\(([^)]*)\)", code)
    assert calls
    for name, args in calls:
        fn = getattr(pkg, name)
        params = inspect.signature(fn).parameters
        for kw in re.findall(r"(\w+)=", args):
            assert kw in params, (name, kw)
