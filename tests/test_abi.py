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
