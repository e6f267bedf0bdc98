"""The C ABI without a GPU: libgsr.so builds for sm_103a, loads, exports every
function include/gsr.h declares, and the ctypes structures of the binding have
the layout a C compiler gives the header's structs.  No compute call is made.
"""
import ctypes as C
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
  printf("%zu\n", offsetof(gsr_config, blend_batch_bwd));
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
    assert sizes[11] == L.Config.blend_batch_bwd.offset
    assert sizes[12:14] == [C.sizeof(L.InsertParams), L.InsertParams.tau_a.offset]


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
