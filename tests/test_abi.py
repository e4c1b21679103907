"""The C-ABI library loads, exports every entry point include/bdra.h declares,
and rejects bad arguments before touching a device (no GPU needed)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2206_05851_gb300 import bdra, build as B
from paper_2206_05851_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return bdra.load()


def _declared():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(bd_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_method_calls():
    names = _declared()
    for n in ("bd_create", "bd_spawn_replicas", "bd_step", "bd_replica_average",
              "bd_detect_events", "bd_destroy"):
        assert n in names


def test_header_is_plain_c(tmp_path):
    # the boundary is a C ABI: the header compiles as strict C99, without C++
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "t.c"
    src.write_text('#include "bdra.h"\nint main(void) { bd_config c; bd_chain_desc d; '
                   '(void)c; (void)d; return 0; }\n')
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc,
                        "-fsyntax-only", str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_binding_structs_match_the_header(tmp_path):
    # the ctypes mirrors of bd_chain_desc, bd_config, bd_event and bd_info
    # have the C structs' sizes and field offsets
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = [bdra.bd_chain_desc, bdra.bd_config, bdra.bd_event, bdra.bd_info]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "bdra.h"', 'int main(void) {']
    for st in structs:
        lines.append(f'printf("%zu\\n", sizeof({st.__name__}));')
        for f, _ in st._fields_:
            lines.append(f'printf("%zu\\n", offsetof({st.__name__}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run([gcc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = []
    for st in structs:
        want.append(ctypes.sizeof(st))
        want += [getattr(st, f).offset for f, _ in st._fields_]
    assert got == want


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm_103a(lib):
    # the fatbin of an sm_103a build names the architecture
    blob = open(bdra.LIB_PATH, "rb").read()
    assert b"sm_103a" in blob


def test_status_strings(lib):
    assert lib.bd_status_string(0) == b"BD_OK"
    assert lib.bd_status_string(6) == b"BD_E_CAPACITY"
    assert lib.bd_last_error(None) == b"NULL context"


def _cfg(chains, **kw):
    args = dict(dt=1e-3, window_steps=10, seed=0, precision=bdra.BD_PREC_FP32, max_windows=4)
    args.update(kw)
    return bdra.make_config(chains, **args)


def _create(cfg, pos):
    out = ctypes.c_void_p()
    st = bdra.load().bd_create(ctypes.byref(cfg), pos.ctypes.data if pos is not None else None,
                               ctypes.byref(out))
    return st, out.value


GOOD = I.Chain(n_beads=10, n_replicas=4, spring=I.SPRING_FENE, flow=I.FLOW_SHEAR, b=50.0,
               rate=1.0)


@pytest.mark.parametrize("field,value", [
    ("n_beads", 1), ("n_beads", 513), ("n_replicas", 0), ("spring", 7), ("flow", 9),
    ("H", 0.0), ("b", -1.0), ("rate", math.nan)])
def test_bad_chain_rejected_without_device(lib, field, value):
    import dataclasses
    ch = dataclasses.replace(GOOD, **{field: value})
    cfg, _keep = _cfg([ch])
    st, ptr = _create(cfg, np.zeros((max(ch.n_beads, 1), 3)))
    assert st == bdra.BD_E_INVALID and ptr is None


@pytest.mark.parametrize("kw", [dict(dt=0.0), dict(window_steps=0), dict(precision=5),
                                dict(max_windows=-1), dict(s_min=0.0), dict(thr_mask=8),
                                dict(flags=8), dict(lanes_hint=3), dict(lanes_hint=2),
                                dict(layout_hint=3),
                                dict(layout_hint=2, precision=bdra.BD_PREC_FP64),
                                dict(layout_hint=2, lanes_hint=13),
                                dict(checkpoint_steps=15), dict(checkpoint_steps=-10),
                                dict(chain_id_base=-1), dict(chain_id_base=2**31 - 1)])
def test_bad_config_rejected_without_device(lib, kw):
    ch = I.Chain(n_beads=100, n_replicas=4, spring=I.SPRING_FENE, b=50.0)
    cfg, _keep = _cfg([ch, ch], **kw)          # two chains: ids base, base + 1
    st, ptr = _create(cfg, np.zeros((200, 3)))
    assert st == bdra.BD_E_INVALID and ptr is None


COLLAPSED = I.Chain(n_beads=12, n_replicas=3, spring=I.SPRING_HARMONIC, H=400.0, r0=2.0, lj_u=1.0,
                    lj_sigma=2.0)


@pytest.mark.parametrize("chain,kw", [
    (dict(r0=-1.0), {}), (dict(lj_sigma=0.0), {}), (dict(lj_u=-1.0), {}),
    (dict(spring=I.SPRING_FENE, lj_u=1.0), {}),                  # pair forces need a rest-length law
    (dict(hi_a=-0.5), {}), (dict(hi_a=1.0, n_beads=65), {}),     # RPY limits
    (dict(hi_a=1.0), dict(checkpoint_steps=10)),                  # no adjoint with RPY
    ({}, dict(checkpoint_steps=10)),                             # no adjoint for collapsed chains
    (dict(spring=I.SPRING_VWF, vwf_fa=6.3, vwf_fb=271.5, vwf_xmax=0.0), {}),
    (dict(spring=I.SPRING_VWF, vwf_fa=-1.0, vwf_fb=271.5, vwf_xmax=3.4), {}),
    (dict(spring=I.SPRING_VWF, vwf_fa=6.3, vwf_fb=math.inf, vwf_xmax=3.4), {})])
def test_bad_model_parameters_rejected_without_device(lib, chain, kw):
    import dataclasses
    ch = dataclasses.replace(COLLAPSED, **chain)
    cfg, _keep = _cfg([ch], **kw)
    st, ptr = _create(cfg, np.zeros((ch.n_beads, 3)))
    assert st == bdra.BD_E_INVALID and ptr is None


def test_null_arguments_rejected(lib):
    cfg, _keep = _cfg([GOOD])
    st, _ = _create(cfg, None)
    assert st == bdra.BD_E_INVALID
    assert lib.bd_step(None, 10) == bdra.BD_E_INVALID
    assert lib.bd_spawn_replicas(None) == bdra.BD_E_INVALID
    lib.bd_destroy(None)    # NULL is ignored


def test_probe_rejects_null_output(lib):
    assert lib.bd_probe_philox_rounds(None, None) == bdra.BD_E_INVALID
    assert lib.bd_probe_fp32_fma(None, None) == bdra.BD_E_INVALID
    assert lib.bd_probe_fp64_fma(None, None) == bdra.BD_E_INVALID
    assert lib.bd_probe_mufu(None, None) == bdra.BD_E_INVALID
    assert lib.bd_probe_issue(None, None) == bdra.BD_E_INVALID
    assert lib.bd_probe_int_alu(None, None) == bdra.BD_E_INVALID


def test_binding_fails_loudly_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(bdra, "_lib", None)
    monkeypatch.setattr(bdra, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        bdra.load()
