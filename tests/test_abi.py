"""The C ABI library loads and exports what include/fewha.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fewha.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(fewha_[A-Za-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def L():
    from paper_2202_11945_gb300 import build, fewha
    if not os.path.exists(fewha.LIB_PATH):
        build.build()
    return fewha.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert "fewha_reconstruct" in names and "fewha_create" in names
    for n in names:
        assert hasattr(L, n), n


def test_binding_covers_every_export():
    from paper_2202_11945_gb300 import fewha
    assert sorted(fewha.EXPORTS) == _declared()


def _create(L, wl, precision=32):
    from paper_2202_11945_gb300 import fewha
    tel, wfs, layers, dms, params = fewha.structs_from_workload(wl, precision)
    h = ctypes.c_void_p()
    rc = L.fewha_create(ctypes.byref(tel), wfs, len(wfs), layers, len(layers), dms, len(dms),
                        ctypes.byref(params), ctypes.byref(h))
    return rc, h, L.fewha_create_error().decode()


def test_geometry_errors_are_reported_before_any_device_work(L):
    wl = synth.tiny_scao()
    wl["layers"][1]["n"] = 8                     # 8 km footprint needs > 8 nodes
    rc, h, msg = _create(L, wl)
    assert rc == -2 and not h.value and "layer 1" in msg
    wl = synth.tiny_scao()
    wl["layers"][0]["n"] = 24                    # not a power of two
    assert _create(L, wl)[0] == -2
    wl = synth.tiny_scao()
    wl["layers"][0]["levels"] = 6                # more levels than log2(32)
    assert _create(L, wl)[0] == -2
    wl = synth.tiny_mcao()
    wl["wfs"][0]["nb"] = 2                       # coarse LGS
    assert _create(L, wl)[0] == -2
    wl = synth.tiny_scao()
    wl["dms"][0]["spacing"] = 1.2                # DM wider than the ground layer grid
    assert _create(L, wl)[0] == -2


def test_limits_and_bad_arguments(L):
    wl = synth.tiny_scao()
    wl["params"]["iters"] = 1000
    assert _create(L, wl)[0] == -6
    wl = synth.tiny_scao()
    assert _create(L, wl, precision=16)[0] == -1
    wl = synth.tiny_scao()
    wl["wfs"][0]["n_sub"] = 200
    assert _create(L, wl)[0] == -6
    wl = synth.tiny_scao()
    wl["wfs"][0]["sigma"] = 0.0
    assert _create(L, wl)[0] == -1


def test_maory_geometry_passes_validation(L):
    """Validation succeeds; without a GPU, creation stops at the device step."""
    import torch
    rc, h, msg = _create(L, synth.maory())
    if torch.cuda.is_available():
        assert rc == 0
        L.fewha_destroy(h)
    else:
        assert rc == -4 and "device" in msg


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structures of the binding have the C header's sizes and field offsets
    (compiled here with the host C compiler from include/fewha.h)."""
    import shutil
    import subprocess
    from paper_2202_11945_gb300 import fewha
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"fewha_telescope": fewha.Telescope, "fewha_wfs": fewha.Wfs, "fewha_layer": fewha.Layer,
               "fewha_dm": fewha.Dm, "fewha_params": fewha.Params, "fewha_batch_config": fewha.BatchConfig,
               "fewha_lsfit": fewha.LsFit}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fewha.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
