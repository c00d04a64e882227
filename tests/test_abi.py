"""CPU checks of the C-ABI boundary: the library loads, exports every entry
point declared in include/lbm.h, its structs match the binding's layout, and
its host-side eye builder reproduces the oracle's mask bit for bit."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2102_12663_gb300 import _build, lbm
from paper_2102_12663_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def L():
    _build.build()
    return lbm.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point(L):
    names = declared_functions()
    assert "lbm_step" in names and "lbm_create_domain" in names
    for n in names:
        assert hasattr(L, n), f"{n} declared in lbm.h but not exported"


def test_struct_layout_matches_header(tmp_path):
    structs = {"lbm_geometry_desc": lbm.GeometryDesc, "lbm_geometry_info": lbm.GeometryInfo,
               "lbm_params": lbm.Params, "lbm_observables": lbm.Observables,
               "lbm_launch": lbm.Launch, "lbm_vortex_info": lbm.VortexInfo}
    body = "".join(f'printf("{k} %zu\\n", sizeof({k}));' for k in structs)
    fields = [("lbm_params", "seed"), ("lbm_params", "p_sc_pa"), ("lbm_observables", "nan_flag"),
              ("lbm_geometry_desc", "chamber_angle_deg"), ("lbm_geometry_desc", "host_mask"),
              ("lbm_geometry_info", "arc_xc"), ("lbm_params", "h_tm"),
              ("lbm_observables", "u_seep"), ("lbm_launch", "stepping"), ("lbm_launch", "sweep_lag"),
              ("lbm_vortex_info", "max_mm"), ("lbm_vortex_info", "n_fluid"),
              ("lbm_params", "bouzidi"), ("lbm_geometry_info", "arc_r")]
    body += "".join(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));' for s, f in fields)
    body += 'printf("STEP_FLOW %d\\n", LBM_STEP_FLOW);printf("STEP_PER_LAUNCH %d\\n", LBM_STEP_PER_LAUNCH);'
    c = tmp_path / "probe.c"
    c.write_text(f'#include <stdio.h>\n#include <stddef.h>\n#include "lbm.h"\nint main(void){{{body}return 0;}}\n')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(c), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for k, cls in structs.items():
        assert int(out[k]) == ctypes.sizeof(cls), k
    for s, f in fields:
        assert int(out[f"{s}.{f}"]) == getattr(structs[s], f).offset, f"{s}.{f}"
    assert int(out["STEP_FLOW"]) == lbm.STEP_FLOW
    assert int(out["STEP_PER_LAUNCH"]) == lbm.STEP_PER_LAUNCH


@pytest.mark.parametrize("nx,ny,angle", [(160, 80, 45.0), (320, 160, 20.0), (512, 256, 33.3),
                                         (150, 75, 45.0), (1024, 512, 27.5), (4096, 2048, 45.0)])
def test_eye_mask_matches_oracle(L, nx, ny, angle):
    m_lib, info = lbm.build_mask(dict(nx=nx, ny=ny, angle_deg=angle))
    m_orc, g = O.eye_mask(nx, ny, angle)
    assert np.array_equal(m_lib, m_orc)
    assert info["inlet_lo"] == g.inlet_lo and info["inlet_width"] == g.inlet_width
    assert info["arc_xc"] == g.arc_xc and info["arc_yc"] == g.arc_yc
    assert info["n_active"] == int(((m_orc == 0) | (m_orc == 1)).sum())


def test_mask_validation(L):
    m, d = W.channel(8, 4)
    d = dict(d)
    d["periodic_x"] = 0  # fluid touches the left/right edge: must be rejected
    with pytest.raises(lbm.LBMError) as e:
        lbm.build_mask(dict(mask=m, **{k: v for k, v in d.items() if k not in ("nx", "ny")}))
    assert e.value.status == lbm.EINVAL
    with pytest.raises(lbm.LBMError):
        lbm.build_mask(dict(nx=160, ny=40, angle_deg=89.0))  # arc taller than the grid
    bad = np.full((4, 4), 9, dtype=np.uint8)
    with pytest.raises(lbm.LBMError):
        lbm.build_mask(dict(mask=bad))
    solid = np.full((6, 6), 4, dtype=np.uint8)
    with pytest.raises(lbm.LBMError):
        lbm.build_mask(dict(mask=solid))


def test_domain_bytes_and_no_gpu_needed_for_sizes(L):
    g, _ = lbm.geometry_desc(dict(nx=4096, ny=2048, angle_deg=45.0))
    b32 = L.lbm_domain_bytes(ctypes.byref(g), lbm.F32)
    b16 = L.lbm_domain_bytes(ctypes.byref(g), lbm.F16DEV)
    b64 = L.lbm_domain_bytes(ctypes.byref(g), lbm.F64)
    N = 4096 * 2048
    # populations (13 x 4 B), velocity snapshot (2 x 4 B), mask (1 B), an
    # edge-cell entry and its neighbour-type word (2 x 4 B) and room for one
    # edge-cell chunk per 32 cells in the tile list (0.5 B) per cell, plus
    # per-tile tables (tile list, partials, neighbour lists, progress words,
    # sweep items, edge offsets)
    assert 69 * N < b32 < 69 * N + (32 << 20)
    assert b16 < b32 < b64
    assert L.lbm_domain_bytes(ctypes.byref(g), 7) == 0
