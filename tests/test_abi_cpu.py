"""CPU-only checks of the C ABI library: it builds, loads, exports every
declared entry point, and its host-only layout arithmetic matches the sizes
the paper prints (Sections 5, 6.1, 6.3)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(vdi_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_2206_08660_gb300 as V

    return V.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 12, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    import paper_2206_08660_gb300 as V

    for i, name in enumerate(V.STATUS):
        assert lib.vdi_status_str(i).decode() == name


def _golden():
    out = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_sizes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v, unit = line.split()[:3]
        out[k] = float(v) * {"MiB": 2**20, "MB": 2**20}[unit]  # the paper's "MB" at 1024^2 is binary
    return out


@pytest.mark.parametrize("key,w,h", [("vdi_fp32_1280x720_ns20", 1280, 720),
                                     ("vdi_fp32_1920x1080_ns20", 1920, 1080),
                                     ("vdi_fp32_1024x1024_ns20", 1024, 1024)])
def test_layout_matches_paper_vdi_sizes(key, w, h):
    import paper_2206_08660_gb300 as V

    d = V.desc(w, h, 20, np.eye(4), np.eye(4), (0, 0, 0), (1, 1, 1), 1.0, V.VDI_F32)
    L = V.vdi_layout_bytes(d)
    # 24 B per slot, as in the paper's two textures
    assert L.paper_bytes == w * h * 20 * 24
    assert abs(L.paper_bytes / _golden()[key] - 1) < 2e-3
    # the FP32 device layout holds exactly those bytes too (16 B colour + 8 B depth per slot)
    assert L.depth_bytes + L.colour_bytes == L.paper_bytes
    assert L.list_bytes == w * h * 8 + (-(-w // 4)) * (-(-h // 4)) * 8 and L.total_bytes == L.paper_bytes + L.grid_bytes + L.list_bytes
    d16 = V.desc(w, h, 20, np.eye(4), np.eye(4), (0, 0, 0), (1, 1, 1), 1.0, V.VDI_F16)
    L16 = V.vdi_layout_bytes(d16)
    assert L16.depth_bytes + L16.colour_bytes == w * h * 20 * 16


def test_grid_size_matches_paper():
    import paper_2206_08660_gb300 as V

    d = V.desc(1920, 1080, 20, np.eye(4), np.eye(4), (0, 0, 0), (1, 1, 1), 1.0)
    L = V.vdi_layout_bytes(d)
    assert (L.grid_w, L.grid_h, L.grid_nz) == (240, 135, 20)
    assert abs(L.grid_bytes / _golden()["grid_1920x1080"] - 1) < 0.02


def test_layout_rejects_bad_descriptors():
    import paper_2206_08660_gb300 as V

    for bad in [dict(n_s=0), dict(n_s=65), dict(w=0), dict(length_unit=0.0), dict(colour_fmt=7)]:
        kw = dict(w=8, h=8, n_s=4, length_unit=1.0, colour_fmt=V.VDI_F32)
        kw.update(bad)
        d = V.desc(kw["w"], 8, kw["n_s"], np.eye(4), np.eye(4), (0, 0, 0), (1, 1, 1), kw["length_unit"],
                   kw["colour_fmt"])
        with pytest.raises(V.VdiError) as e:
            V.vdi_layout_bytes(d)
        assert e.value.status == 1
    # odd N_S is stored rounded up to even
    assert V.vdi_layout_bytes(V.desc(8, 8, 5, np.eye(4), np.eye(4), (0, 0, 0), (1, 1, 1), 1.0)).n_s_stored == 6


def test_ctypes_structures_match_the_header(tmp_path):
    """Every structure the binding passes across the ABI has the header's
    layout: a C program built against include/vdi.h prints the size of each
    struct and the offset of each field, and the ctypes mirrors must agree."""
    import shutil
    import subprocess

    import paper_2206_08660_gb300 as V

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [("vdi_camera", V.VdiCamera), ("vdi_desc", V.VdiDesc), ("vdi_layout", V.VdiLayout),
             ("vdi_stats_t", V.VdiStats), ("vdi_volume", V.VdiVolume), ("vdi_tf", V.VdiTf),
             ("vdi_gen_params", V.VdiGenParams), ("vdi_request", V.VdiRequest), ("vdi_batch_opts", V.VdiBatchOpts),
             ("vdi_server_config", V.VdiServerConfig), ("vdi_view_request", V.VdiViewRequest),
             ("vdi_ticket_info", V.VdiTicketInfo), ("vdi_server_counters", V.VdiServerCounters),
             ("vdi_render_opts", V.VdiRenderOpts), ("vdi_pi_config", V.VdiPiConfig)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vdi.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for cname, py in pairs:
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
