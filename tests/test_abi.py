"""The C ABI without a GPU: libgsr.so builds for sm_103a, loads, exports every
function include/gsr.h declares, and the ctypes structures of the binding have
the layout a C compiler gives the header's structs.  No compute call is made.
"""
import ctypes as C
import math
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsr.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gsr_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2512_08498_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("gsr_create", "gsr_destroy", "gsr_forward", "gsr_backward", "gsr_tune", "gsr_check",
                     "gsr_debug_lists", "gsr_debug_records", "gsr_debug_pixels", "gsr_saved_create"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_2512_08498_gb300 import _lib
    bound = {name for name, _, _ in _lib.SIGNATURES}
    assert set(_declared_functions()) <= bound, set(_declared_functions()) - bound


def test_struct_layout_matches_c(lib):
    from paper_2512_08498_gb300 import _lib as L
    probe = r"""
#include <stdio.h>
#include <stddef.h>
#include "gsr.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(gsr_config), sizeof(gsr_gaussians), sizeof(gsr_view),
         sizeof(gsr_outputs), sizeof(gsr_grads), sizeof(gsr_saved_info));
  printf("%zu %zu %zu\n", offsetof(gsr_view, viewmat), offsetof(gsr_view, subset), offsetof(gsr_view, subset_count));
  printf("%zu %zu\n", offsetof(gsr_config, near_plane), offsetof(gsr_config, flags));
  printf("%zu %zu\n", offsetof(gsr_config, blend_batch_bwd), offsetof(gsr_config, list_prefix));
  printf("%zu %zu %zu\n", offsetof(gsr_saved_info, list_prefix), offsetof(gsr_saved_info, open_tiles),
         offsetof(gsr_saved_info, list_span));
  printf("%zu %zu\n", sizeof(gsr_insert_params), offsetof(gsr_insert_params, tau_a));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(src, "w").write(probe)
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    sizes = [int(x) for x in out]
    assert sizes[:6] == [C.sizeof(L.Config), C.sizeof(L.Gaussians), C.sizeof(L.View), C.sizeof(L.Outputs),
                         C.sizeof(L.Grads), C.sizeof(L.SavedInfo)]
    assert sizes[6:9] == [L.View.viewmat.offset, L.View.subset.offset, L.View.subset_count.offset]
    assert sizes[9:11] == [L.Config.near_plane.offset, L.Config.flags.offset]
    assert sizes[11:13] == [L.Config.blend_batch_bwd.offset, L.Config.list_prefix.offset]
    assert sizes[13:16] == [L.SavedInfo.list_prefix.offset, L.SavedInfo.open_tiles.offset,
                            L.SavedInfo.list_span.offset]
    assert sizes[16:18] == [C.sizeof(L.InsertParams), L.InsertParams.tau_a.offset]


def test_non_compute_calls(lib):
    from paper_2512_08498_gb300 import _lib as L
    l = L.load()
    assert l.gsr_version().decode().startswith("gsr")
    cfg = L.Config()
    l.gsr_config_default(C.byref(cfg))
    assert (cfg.tile_w, cfg.tile_h, cfg.blend_batch, cfg.sh_degree) == (16, 16, 256, 3)
    assert cfg.blend_batch_bwd == 128
    assert abs(cfg.near_plane - 0.2) < 1e-7
    # invalid arguments are rejected before any device work
    assert l.gsr_create(None, C.byref(cfg)) == L.GSR_ERR_INVALID_ARG
    bad = L.Config()
    l.gsr_config_default(C.byref(bad))
    bad.tile_w = 12
    h = C.c_void_p()
    assert l.gsr_create(C.byref(h), C.byref(bad)) == L.GSR_ERR_INVALID_ARG
    l.gsr_config_default(C.byref(bad))
    bad.blend_batch_bwd = 100
    assert l.gsr_create(C.byref(h), C.byref(bad)) == L.GSR_ERR_INVALID_ARG
    assert cfg.list_prefix == 1.0   # one list round by default
    for v in (-0.5, float("nan"), float("inf")):
        l.gsr_config_default(C.byref(bad))
        bad.list_prefix = v
        assert l.gsr_create(C.byref(h), C.byref(bad)) == L.GSR_ERR_INVALID_ARG
    assert l.gsr_l1_loss_grad(None, None, -1, None, None, None) == L.GSR_ERR_INVALID_ARG
    ip = L.InsertParams()
    l.gsr_insert_params_default(C.byref(ip))
    assert abs(ip.sigma - 1.0) < 1e-7 and abs(ip.tau_a - 0.2) < 1e-7
    assert l.gsr_insertion(None, C.byref(ip), None, 1, None, None, None, None, None, None, 0, None,
                           None) == L.GSR_ERR_INVALID_ARG
    assert l.gsr_rig_chain(None, 1, None, None, None, None, None, 1, 0, None, None, None,
                           None) == L.GSR_ERR_INVALID_ARG
    assert l.gsr_dft_energy(None, None, 1, None, None) == L.GSR_ERR_INVALID_ARG
    assert l.gsr_frequency_schedule(None, 1, None, None, None, 2.0, None, 0, None, None, None, None,
                                    None) == L.GSR_ERR_INVALID_ARG
    assert C.sizeof(L.Image) == 24
    mp = L.MergeParams()
    l.gsr_merge_params_default(C.byref(mp))
    assert abs(mp.tau_d - 0.5) < 1e-7 and abs(mp.near_plane - 0.2) < 1e-7
    assert l.gsr_merge(None, C.byref(mp), None, 0, None, None, None, 3, 0, None, None, None, None, None,
                       None) == L.GSR_ERR_INVALID_ARG
    assert C.sizeof(L.MergeOutputs) == 56


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_2512_08498_gb300 import _lib as L
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        L._lib_saved = L._lib
        try:
            L._lib = None
            L.load(str(tmp_path / "missing.so"))
        finally:
            L._lib = L._lib_saved


def _choice(l, sat, inst, visible):
    from paper_2512_08498_gb300 import _lib as L
    H = (C.c_uint64 * (L.GSR_LIST_BUCKETS + 1))(*[int(x) for x in sat])
    J = (C.c_uint64 * L.GSR_LIST_BUCKETS)(*[int(x) for x in inst])
    return l.gsr_list_prefix_choice(C.cast(H, C.c_void_p), C.cast(J, C.c_void_p), visible)


def test_automatic_list_rule(lib):
    """The host rule of the automatic list mode on constructed histograms: the
    edges are geometric, a batch whose tiles all saturate within the nearest
    few records takes two rounds with a first round just past the last
    saturating bucket, one whose tiles need most records (or never saturate)
    takes one, and no measurement keeps the previous choice."""
    from paper_2512_08498_gb300 import _lib as L
    l = L.load()
    nb = L.GSR_LIST_BUCKETS
    edges = [l.gsr_list_bucket_edge(b) for b in range(nb + 1)]
    assert abs(edges[0] - 2.0 ** -12) < 1e-15 and edges[nb] == 1.0
    ratios = [edges[b + 1] / edges[b] for b in range(nb)]
    assert max(ratios) - min(ratios) < 1e-12
    # instances spread by depth share like a single dense view: a record's
    # instances in proportion to the records' share of the bucket
    inst = [0] * nb
    for b in range(nb):
        inst[b] = 1000 * (edges[b + 1] - edges[b]) * 74_000
    # every tile saturates within buckets <= 10
    sat = [0] * (nb + 1)
    sat[8], sat[10] = 40_000_000, 34_000_000
    f = _choice(l, sat, inst, 500_000)
    assert 0 < f < 1 and abs(f - edges[11]) < 1e-6, f
    # tiles that need almost every record: one round
    sat = [0] * (nb + 1)
    sat[nb - 1] = 74_000_000
    assert _choice(l, sat, inst, 500_000) == 1.0
    # like the rig: near records hold most instances (cumulative share of
    # instances ~ sqrt of the share of records) and the tiles saturate
    # spread over 30-90 % of the records: one round
    front = [19_400_000 * (math.sqrt(edges[b + 1]) - math.sqrt(edges[b])) for b in range(nb)]
    sat = [0] * (nb + 1)
    for b in range(50, 63):
        sat[b] = 19_400_000 // 13
    assert _choice(l, sat, front, 1_470_000) == 1.0
    # most of the lists in tiles that never saturate: one round
    sat = [0] * (nb + 1)
    sat[8], sat[nb] = 10_000_000, 64_000_000
    assert _choice(l, sat, inst, 500_000) == 1.0
    # many records per instance and a few tiles that never saturate: the
    # second round's walk over every record costs most of a round, so one
    sat = [0] * (nb + 1)
    sat[10], sat[nb] = 73_000_000, 1_000_000
    assert _choice(l, sat, inst, 200_000_000) == 1.0
    # the same without the open tiles: the first round walks few records
    # and the second has nothing to do, so two
    sat[10], sat[nb] = 74_000_000, 0
    assert abs(_choice(l, sat, inst, 200_000_000) - edges[11]) < 1e-6
    # no instance histogram: no measurement
    assert _choice(l, sat, [0] * nb, 500_000) == -1.0
    assert l.gsr_list_prefix_choice(None, None, 0) == -1.0
