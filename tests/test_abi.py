"""The C-ABI library builds, loads and exports every entry point the header
declares, and the binding's struct layouts match the header's. CPU only (no
compute calls)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ngs.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"NGS_API\s+[\w\s\*]+?\b(ngs_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_15186_gb300 import build
    path = build.build()
    return C.CDLL(path), path


def test_header_declares_the_boundary():
    names = _declared()
    for want in ["ngs_create", "ngs_load_scene", "ngs_select_cut", "ngs_render", "ngs_destroy",
                 "ngs_strerror", "ngs_sort_pairs", "ngs_scan_u32"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    L, path = lib
    for name in _declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ngs_\w+)", out))
    assert set(_declared()) <= exported
    # nothing else of the renderer leaks out of the library
    assert exported == set(_declared())


def test_binding_covers_every_declared_symbol():
    from paper_2603_15186_gb300 import _lib
    assert sorted(_lib.EXPORTS) == _declared()


def test_strerror_without_gpu(lib):
    L, _ = lib
    L.ngs_strerror.restype = C.c_char_p
    assert L.ngs_strerror(0) == b"ok"
    assert L.ngs_strerror(4) == b"work buffer capacity exceeded"


def test_struct_layouts_match_header(tmp_path):
    from paper_2603_15186_gb300 import _lib
    prog = tmp_path / "layout.c"
    prog.write_text(r"""
#include <stdio.h>
#include <stddef.h>
#include "ngs.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(ngs_camera), sizeof(ngs_gaussians),
         sizeof(ngs_hierarchy), sizeof(ngs_config), sizeof(ngs_stats));
  printf("%zu %zu %zu %zu\n", offsetof(ngs_camera, tau), offsetof(ngs_gaussians, attr_dtype),
         offsetof(ngs_config, max_tiles_per_batch), offsetof(ngs_stats, mode));
  printf("%zu %zu %zu %zu %zu %d %zu %zu\n", sizeof(ngs_tune_result), offsetof(ngs_tune_result, ms),
         offsetof(ngs_tune_result, batch), offsetof(ngs_stats, cta_w), sizeof(ngs_server_config),
         NGS_TUNE_SHAPES, sizeof(ngs_slice_grid), offsetof(ngs_slice_grid, threshold));
  printf("%d %d %d %d %d %d %d %d %d %d %d %d %d %zu\n", NGS_OPT_MODE, NGS_OPT_TILE_W,
         NGS_OPT_TILE_H, NGS_OPT_BATCH, NGS_OPT_GRAPH, NGS_OPT_STAGE_TIMING, NGS_OPT_BLOCK_CULL,
         NGS_OPT_CTA_W, NGS_OPT_CTA_H, NGS_OPT_PAIRS_PER_PIXEL, NGS_OPT_LOD_BLEND,
         NGS_OPT_COMPOSITE_ORDER, NGS_OPT_NODE_IDS, offsetof(ngs_stats, composite_tail_ms));
  printf("%d\n", NGS_CUT_FRUSTUM);
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    a, b, t, o, f = subprocess.run([str(exe)], capture_output=True, text=True,
                                   check=True).stdout.split("\n")[:5]
    sizes = [int(x) for x in a.split()]
    offs = [int(x) for x in b.split()]
    assert sizes == [C.sizeof(_lib.Camera), C.sizeof(_lib.Gaussians), C.sizeof(_lib.Hierarchy),
                     C.sizeof(_lib.Config), C.sizeof(_lib.Stats)]
    assert offs == [_lib.Camera.tau.offset, _lib.Gaussians.attr_dtype.offset,
                    _lib.Config.max_tiles_per_batch.offset, _lib.Stats.mode.offset]
    assert [int(x) for x in t.split()] == [
        C.sizeof(_lib.TuneResult), _lib.TuneResult.ms.offset, _lib.TuneResult.batch.offset,
        _lib.Stats.cta_w.offset, C.sizeof(_lib.ServerConfig), len(_lib.TUNE_SHAPES),
        C.sizeof(_lib.SliceGrid), _lib.SliceGrid.threshold.offset]
    assert [int(x) for x in o.split()] == [
        _lib.NGS_OPT_MODE, _lib.NGS_OPT_TILE_W, _lib.NGS_OPT_TILE_H, _lib.NGS_OPT_BATCH,
        _lib.NGS_OPT_GRAPH, _lib.NGS_OPT_STAGE_TIMING, _lib.NGS_OPT_BLOCK_CULL,
        _lib.NGS_OPT_CTA_W, _lib.NGS_OPT_CTA_H, _lib.NGS_OPT_PAIRS_PER_PIXEL,
        _lib.NGS_OPT_LOD_BLEND, _lib.NGS_OPT_COMPOSITE_ORDER, _lib.NGS_OPT_NODE_IDS,
        _lib.Stats.composite_tail_ms.offset]
    assert int(f) == _lib.CUT_FRUSTUM


def test_renderer_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2603_15186_gb300 import Renderer, NgsError
    with pytest.raises((NgsError, RuntimeError)):
        Renderer(device=0)


def test_rect_packing_round_trips_at_its_limits(tmp_path):
    """The 8-byte tile rectangle of the binning stages keeps every tile
    coordinate an image of up to 32768 pixels can have with 8-pixel tiles
    (0..4095) and every camera index of a launch (0..65535). Host code of the
    library's own header, compiled by nvcc; no GPU."""
    from paper_2603_15186_gb300 import build
    prog = tmp_path / "rect.cu"
    prog.write_text(r"""
#include <cstdio>
#include "ngs_internal.cuh"
int main() {
  const uint32_t co[] = {0u, 1u, 255u, 256u, 2047u, 4094u, 4095u};
  const uint32_t cams[] = {0u, 1u, 255u, 256u, 1023u, 1024u, 65535u};
  long bad = 0, n = 0;
  for (uint32_t a : co) for (uint32_t b : co) for (uint32_t c : co) for (uint32_t d : co)
    for (uint32_t k : cams) {
      const ngs::RectU u = ngs::unpack_rect(ngs::pack_rect(a, b, c, d, k));
      bad += u.x0 != a || u.y0 != b || u.x1 != c || u.y1 != d || u.cam != k;
      ++n;
    }
  std::printf("%ld %ld %u\n", n, bad, ngs::kRectCoordMax);
  return 0;
}
""")
    exe = tmp_path / "rect"
    subprocess.run([build.nvcc(), "-std=c++17", "-I", os.path.join(ROOT, "include"),
                    "-I", build.CSRC, str(prog), "-o", str(exe)], check=True)
    n, bad, cmax = (int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.split())
    assert n == 7 ** 5 and bad == 0
    # 32768-pixel images in 8-pixel tiles: 4096 tiles per axis
    assert cmax == 32768 // 8
