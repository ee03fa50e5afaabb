"""The C-ABI library builds, loads without a GPU, and exports every function
that include/*.h declares; the ctypes mirrors of the public structs have the
header's sizes and offsets (checked by compiling the header with gcc)."""
import ctypes as C
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def potlib():
    from paper_2103_14024_gb300 import build_lib
    build_lib.build()
    import paper_2103_14024_gb300 as pot
    return pot


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(pot_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_exported(potlib):
    names = _declared_functions()
    assert "pot_render" in names and "pot_build_sparse" in names
    L = C.CDLL(potlib.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_loads_and_reports_without_gpu(potlib):
    assert potlib.lib().pot_version() >= 1
    assert potlib.launch_count() >= 0


def test_struct_layouts_match_header(potlib, tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "pot.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(pot_camera), sizeof(pot_build_desc), sizeof(pot_render_opts),
         sizeof(pot_tree_info));
  printf("%zu %zu %zu\\n", offsetof(pot_render_opts, max_steps), offsetof(pot_render_opts, seg_count),
         offsetof(pot_tree_info, bbox_lo));
  return 0;
}
""")
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    sizes = [int(v) for v in out]
    assert sizes[:4] == [C.sizeof(potlib.Camera), C.sizeof(potlib.BuildDesc), C.sizeof(potlib.RenderOpts),
                         C.sizeof(potlib.TreeInfo)]
    assert sizes[4] == potlib.RenderOpts.max_steps.offset
    assert sizes[5] == potlib.RenderOpts.seg_count.offset
    assert sizes[6] == potlib.TreeInfo.bbox_lo.offset


def test_camera_record_matches_generator(potlib):
    from paper_2103_14024_gb300 import synth
    assert synth.CAMERA_DTYPE.itemsize == C.sizeof(potlib.Camera) == 80
    for name, (dt, off) in synth.CAMERA_DTYPE.fields.items():
        assert getattr(potlib.Camera, name).offset == off


def test_missing_library_fails_loudly(potlib, monkeypatch):
    import importlib
    mod = importlib.import_module("paper_2103_14024_gb300")
    monkeypatch.setattr(mod, "_lib", None)
    monkeypatch.setattr(mod, "LIB_PATH", os.path.join(ROOT, "does-not-exist", "libpot.so"))
    with pytest.raises(RuntimeError):
        mod.lib()


def test_segment_record_constants_match_header(potlib, tmp_path):
    """The record size and slot block of include/pot_segments.h are the binding's,
    and the binding's ctypes signatures of the two recorded-segment calls have
    one argument per parameter of the header's declarations."""
    prog = tmp_path / "seg.c"
    prog.write_text("""
#include <stdio.h>
#include "pot_segments.h"
int main(void) { printf("%d %d\\n", POT_SEGMENT_RECORD_BYTES, POT_SEGMENT_BLOCK); return 0; }
""")
    exe = tmp_path / "seg"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    rec, block = (int(v) for v in subprocess.check_output([str(exe)]).decode().split())
    assert rec == potlib.SEGMENT_RECORD_BYTES == 32
    assert block == potlib.SEGMENT_BLOCK
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "pot_segments.h")).read(), flags=re.S)
    for name in ("pot_render_rays_record", "pot_render_backward_recorded"):
        m = re.search(name + r"\s*\(([^)]*)\)", src)
        assert m, name
        n_params = len([p for p in m.group(1).split(",") if p.strip()])
        assert len(potlib._SIGS[name]) == n_params, name


def test_segment_records_buffer_host_logic(potlib):
    """SegmentRecords sizing: 32-byte rows, a two-int64 state, and room for one
    partly used block of slots per resident warp beyond the expected segments."""
    import torch
    r = potlib.SegmentRecords(1000, device="cpu")
    assert r.records.shape == (1000, 8) and r.records.dtype == torch.float32
    assert r.records.element_size() * r.records.shape[1] == potlib.SEGMENT_RECORD_BYTES
    assert r.state.dtype == torch.int64 and r.state.tolist() == [0, 0]
    assert potlib.SegmentRecords(0, device="cpu").records.shape[0] == 1   # never a zero-size tensor
    big = potlib.SegmentRecords.for_rays(1 << 18, 64, device="cpu")
    assert big.capacity >= (1 << 18) * 64 + 152 * 24 * potlib.SEGMENT_BLOCK   # 152 SMs x 24 resident warps
    assert big.capacity < (1 << 31)
