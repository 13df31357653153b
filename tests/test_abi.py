"""The C-ABI library loads on a CPU-only host and exports every function include/jde.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "jde.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:jde_status|void|int|unsigned long long|const char\s*\*)\s+(jde_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def jde():
    from paper_2011_03910_gb300 import _build
    _build.build()
    from paper_2011_03910_gb300 import jde as j
    return j


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("jde_create", "jde_detect_batch", "jde_track_step", "jde_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(jde):
    for name in declared_functions():
        assert hasattr(jde.lib, name), name
    assert set(declared_functions()) <= set(jde.EXPORTED)


def test_layer_table_matches_oracle(jde):
    from oracle import network as net
    assert jde.jde_layer_table() == net.layer_specs()


def test_default_config_values(jde):
    c = jde.jde_default_config()
    assert (c.precision, c.conf_thresh, c.nms_iou, c.lost_max_frames) == (jde.JDE_BF16, 0.5, pytest.approx(0.4), 30)
    assert c.gate_chi2 == 9.487729036781154 and c.max_cand == 4096


def test_create_rejects_bad_config_without_gpu(jde):
    c = jde.jde_default_config()
    c.max_in_w = 1000          # not a multiple of 32: rejected before any CUDA call
    with pytest.raises(jde.JdeError) as e:
        jde.jde_create(c, b"JDEW")
    assert e.value.status == 1
    jde.jde_destroy(None)      # NULL is a no-op


def test_dependent_launch_option_is_validated_without_gpu(jde):
    c = jde.jde_default_config()
    assert c.dependent_launch == 1 and c.fuse_block1 == 0
    c.dependent_launch = 2     # only 0 or 1: rejected before any CUDA call
    with pytest.raises(jde.JdeError) as e:
        jde.jde_create(c, b"JDEW")
    assert e.value.status == 1
    assert jde.lib.jde_set_dependent_launch(None, 1) == 1     # NULL handle: JDE_ERR_INVALID_ARG


def test_binding_structs_match_the_header_layout(jde, tmp_path):
    """The ctypes structures of the binding have the sizes and field offsets the C compiler gives the
    header's structs (compiled here with gcc against include/jde.h)."""
    import ctypes as C
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = {"jde_config": jde.jde_config, "jde_layer_desc": jde.jde_layer_desc, "jde_dets": jde.jde_dets,
               "jde_tracks": jde.jde_tracks}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "jde.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            parts = line.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
