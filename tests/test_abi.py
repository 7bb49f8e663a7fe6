"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/m2m.h declares; argument validation needs no GPU."""
import ctypes
import os
import re

import numpy as np

import pytest

from paper_1207_6403_gb300 import m2m as B

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "m2m.h")


def declared():
    txt = open(HDR).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(m2m_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared()
    for required in ("m2m_init", "m2m_step", "m2m_observe", "m2m_update_weights",
                     "m2m_priors", "m2m_potential", "m2m_free"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = B.library()
    for name in declared():
        assert hasattr(L, name), name


def test_struct_layouts_match_header_sizes():
    assert ctypes.sizeof(B.m2m_potential_desc) == 40
    assert ctypes.sizeof(B.m2m_obs_desc) == 88
    assert ctypes.sizeof(B.m2m_prior_desc) == 32
    assert ctypes.sizeof(B.m2m_params) == 56
    assert ctypes.sizeof(B.m2m_record) == 56


def _init(**kw):
    L = B.library()
    P = ctypes.c_void_p
    args = dict(prec=B.FP32C, n=100, ptrs=[P(1 << 20)] * 8, nsets=1, par=B.m2m_params(0, 0, 0.01, 0.5, 1, 0, 1))
    args.update(kw)
    ex = (ctypes.c_double * 3)(0.0, 1.0, 2.0)
    od = (B.m2m_obs_desc * 1)()
    od[0].geom, od[0].quant, od[0].nx, od[0].ny = 1, 1, 2, 1
    od[0].edges_x = ctypes.cast(ex, ctypes.POINTER(ctypes.c_double))
    ctx = P()
    pots = args.get("pots", [])
    pd = (B.m2m_potential_desc * max(1, len(pots)))()
    for k, (kind, prm) in enumerate(pots):
        pd[k].kind = kind
        for j, v in enumerate(prm):
            pd[k].p[j] = v
    rc = L.m2m_init(ctypes.byref(ctx), args["prec"], args["n"], *args["ptrs"], pd if pots else None, len(pots), od,
                    args["nsets"], None, None, ctypes.byref(args["par"]), None, None)
    return rc, ctx, L.m2m_last_error(None).decode()


@pytest.mark.parametrize("kw,needle", [
    (dict(prec=7), "precision"),
    (dict(n=0), "n="),
    (dict(ptrs=[ctypes.c_void_p(1 << 20)] * 7 + [ctypes.c_void_p((1 << 20) + 8)]), "aligned"),
    (dict(ptrs=[None] + [ctypes.c_void_p(1 << 20)] * 7), "NULL"),
    (dict(nsets=0), "nsets"),
    (dict(par=B.m2m_params(0, 0, 0.01, 0.0, 1, 0, 1)), "alpha"),
    (dict(par=B.m2m_params(float("nan"), 0, 0.01, 0.5, 1, 0, 1)), "non-finite"),
    (dict(pots=[(4, (2, 1e-3, 100.0, 50))]), "sh needs"),
    (dict(pots=[(4, (256.5, 1e-3, 100.0, 50))]), "sh needs"),
    (dict(pots=[(4, (256, 1.0, 0.5, 50))]), "sh needs"),
    (dict(pots=[(4, (256, 1e-3, 100.0, 0))]), "sh needs"),
    (dict(pots=[(4, (1024, 1e-3, 100.0, 50))]), "sh needs"),
    (dict(pots=[(4, (256, 1e-3, 100.0, 50)), (1, (1.0, 1.0))]), "must be last"),
    (dict(pots=[(9, (1.0, 1.0))]), "unknown potential"),
])
def test_init_rejects_bad_arguments_without_touching_memory(kw, needle):
    rc, ctx, msg = _init(**kw)
    assert rc == -1 and not ctx.value
    assert needle in msg


def test_null_context_is_an_argument_error():
    L = B.library()
    assert L.m2m_set_lazy_update(None, 1) == -1
    assert L.m2m_finish_update(None) == -1
    assert L.m2m_get_record_async(None, None) == -1
    assert L.m2m_step(None, 1) == -1
    assert L.m2m_free(None) == 0


@pytest.mark.parametrize("entries,ncell,needle", [
    ([0, 1, 2, 5], 3, "lookup-table entry 3 = 5"),
    ([0, -2, 1, 1], 3, "lookup-table entry 1 = -2"),
    ([0, 1, 1, 0], 0, "bad geometry"),
    (None, 3, "bad geometry"),
])
def test_lut_sets_are_checked_before_any_device_work(entries, ncell, needle):
    """A 2 x 2 pixel lookup-table set: every entry must name an aperture of
    the set or -1; the table and a positive aperture count are required."""
    L = B.library()
    P = ctypes.c_void_p
    e = (ctypes.c_double * 3)(0.0, 1.0, 2.0)
    od = (B.m2m_obs_desc * 1)()
    od[0].geom, od[0].quant, od[0].nx, od[0].ny = 4, 1, 2, 2
    od[0].edges_x = ctypes.cast(e, ctypes.POINTER(ctypes.c_double))
    od[0].edges_y = ctypes.cast(e, ctypes.POINTER(ctypes.c_double))
    if entries is not None:
        lut = (ctypes.c_int32 * 4)(*entries)
        od[0].lut = ctypes.cast(lut, ctypes.POINTER(ctypes.c_int32))
    od[0].ncell = ncell
    ctx = P()
    par = B.m2m_params(0, 0, 0.01, 0.5, 1, 0, 1)
    rc = L.m2m_init(ctypes.byref(ctx), B.FP32C, 100, *([P(1 << 20)] * 8), None, 0, od, 1, None, None,
                    ctypes.byref(par), None, None)
    assert rc == -1 and not ctx.value
    assert needle in L.m2m_last_error(None).decode()


def test_batch_record_gather_rejects_null():
    L = B.library()
    assert L.m2m_batch_get_records(None, None) == -1


def test_velocity_moments_rejects_null():
    L = B.library()
    assert L.m2m_velocity_moments(None, None, 1, None) == -1


def test_struct_field_offsets_match_the_header(tmp_path):
    """Every field of every structure the binding passes has the offset and
    the structure the size that a C compiler gives the header's definition
    (gcc on the host: the layout rules of the C ABI)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [B.m2m_potential_desc, B.m2m_obs_desc, B.m2m_prior_desc, B.m2m_params, B.m2m_tuning,
               B.m2m_timing, B.m2m_model_desc, B.m2m_record]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "m2m.h"', "int main(void) {"]
    for S in structs:
        name = S.__name__
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in S._fields_:
            lines.append(f'printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "offsets.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "offsets"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)])
    got = {}
    for ln in subprocess.check_output([str(exe)], text=True).splitlines():
        s, f, v = ln.split()
        got[(s, f)] = int(v)
    for S in structs:
        assert got[(S.__name__, "size")] == ctypes.sizeof(S), S.__name__
        for f in S._fields_:
            assert got[(S.__name__, f[0])] == getattr(S, f[0]).offset, (S.__name__, f[0])


def test_seeing_tables_marshal_with_their_bit_count():
    from paper_1207_6403_gb300 import inputs as I
    ex = I.uniform_edges(4, -1.0, 1.0)
    keep = []
    od = B._obs_array([I.ObservableSet("grid", "mass", ex, ex.copy(), psf_q=np.zeros(64), psf_seed=7)], keep)
    assert od[0].psf_bits == 6 and od[0].psf_seed == 7 and od[0].geom == 3
    with pytest.raises(ValueError):
        B._obs_array([I.ObservableSet("grid", "mass", ex, ex.copy(), psf_q=np.zeros(48))], [])
    lut = np.array([[0, 1, -1, 2]] * 4, np.int32)
    od = B._obs_array([I.ObservableSet("lut", "gh", ex, ex.copy(), gh_V=np.zeros(3), gh_S=np.ones(3),
                                       lut=lut, n_apertures=3)], keep)
    assert od[0].geom == 4 and od[0].ncell == 3 and od[0].nx == 4 and od[0].ny == 4
    assert [od[0].lut[k] for k in range(4)] == [0, 1, -1, 2]


def test_philox_entry_rejects_bad_sizes_without_a_gpu():
    L = B.library()
    P = ctypes.c_void_p
    buf = (ctypes.c_uint32 * 8)()
    assert L.m2m_philox4x32_10(0, buf, buf, buf) == -1
    assert L.m2m_philox4x32_10(1, None, buf, buf) == -1
    assert "2^24" in L.m2m_last_error(None).decode()
