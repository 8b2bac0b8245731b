"""The C-ABI library loads and exports every symbol include/rr.h declares,
and the binding's structs match the header's layout.  CPU only: no call
here needs a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rr.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_03505_gb300 import build, rr
    build.build()
    return rr.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2310_03505_gb300 import rr
    assert sorted(rr.SIGNATURES) == declared_functions()
    for n in declared_functions():
        assert callable(getattr(rr, n)), n


def test_struct_layout_matches_header():
    """Compile a probe against the header and compare sizes and offsets."""
    import subprocess
    import tempfile
    from paper_2310_03505_gb300 import rr
    probe = r'''
#include <stdio.h>
#include <stddef.h>
#include "rr.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(rr_material), sizeof(rr_pose), sizeof(rr_sensor_params),
         sizeof(rr_segment), sizeof(rr_scene_info), sizeof(rr_stats), sizeof(rr_profile));
  printf("%zu %zu %zu\n", offsetof(rr_sensor_params, seed), offsetof(rr_sensor_params, scan_id),
         offsetof(rr_sensor_params, flags));
  printf("%zu %zu %zu\n", sizeof(rr_batch_config), offsetof(rr_batch_config, node_format),
         offsetof(rr_batch_config, workspace_limit));
  printf("%zu %zu %zu %zu %zu\n", sizeof(rr_serve_config), sizeof(rr_serve_record), sizeof(rr_serve_stats),
         offsetof(rr_serve_stats, busy_ms), offsetof(rr_serve_record, submit_ms));
  return 0;
}
'''
    d = tempfile.mkdtemp()
    with open(os.path.join(d, "p.c"), "w") as f:
        f.write(probe)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", os.path.join(d, "p"), os.path.join(d, "p.c")],
                   check=True)
    out = subprocess.run([os.path.join(d, "p")], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out[:7]]
    assert sizes == [C.sizeof(rr.rr_material), C.sizeof(rr.rr_pose), C.sizeof(rr.rr_sensor_params),
                     C.sizeof(rr.rr_segment), C.sizeof(rr.rr_scene_info), C.sizeof(rr.rr_stats),
                     C.sizeof(rr.rr_profile)]
    assert [int(x) for x in out[7:10]] == [rr.rr_sensor_params.seed.offset, rr.rr_sensor_params.scan_id.offset,
                                          rr.rr_sensor_params.flags.offset]
    assert [int(x) for x in out[10:13]] == [C.sizeof(rr.rr_batch_config), rr.rr_batch_config.node_format.offset,
                                           rr.rr_batch_config.workspace_limit.offset]
    assert [int(x) for x in out[13:18]] == [C.sizeof(rr.rr_serve_config), C.sizeof(rr.rr_serve_record),
                                           C.sizeof(rr.rr_serve_stats), rr.rr_serve_stats.busy_ms.offset,
                                           rr.rr_serve_record.submit_ms.offset]
    assert rr.SEGMENT_DTYPE.itemsize == C.sizeof(rr.rr_segment)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2310_03505_gb300 import rr
    saved = rr._lib
    rr._lib = None
    try:
        with pytest.raises(RuntimeError):
            rr.load(str(tmp_path / "nope.so"))
    finally:
        rr._lib = saved
