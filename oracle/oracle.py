"""ctypes binding of the CPU reference rasterizer in ``gsr_oracle.c``.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the CPU-baseline leg of the benchmark, never by the product path.  It
imports nothing from the CUDA package; inputs come from plain numpy arrays
(the seeded scene generators produce them).

The oracle follows the 3DGS rasterizer that the paper optimises in Sec. 3.3
(Gaussians and camera poses updated jointly; SH gradients detached for the
camera update):

* ``mirror``    binary32 decision mirror of the preprocess step (culls, radius,
                tile rectangle, depth key bits, colour clamp, blend inputs);
* ``lists``     (view, tile, depth) 64-bit keys sorted with ties by record
                index, and the per-tile ranges;
* ``rec64``     FP64 projected Gaussians (decisions from the mirror);
* ``forward``   per-pixel front-to-back compositing, FP64 values, binary32
                decisions (alpha clamp 0.99, 1/255 skip, 1e-4 stop);
* ``backward``  exact adjoint, including the se(3) camera-pose gradient.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no implicit FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-fvisibility=hidden", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


# ----------------------------------------------------------------------------
# ctypes structures mirroring gsr_oracle.c
# ----------------------------------------------------------------------------

_fp = C.POINTER(C.c_float)
_dp = C.POINTER(C.c_double)
_u32p = C.POINTER(C.c_uint32)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_u64p = C.POINTER(C.c_uint64)


class _Scene(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("sh_degree", C.c_int),
        ("means", _fp), ("log_scales", _fp), ("quats", _fp), ("opac", _fp), ("sh", _fp),
        ("means64", _dp), ("log_scales64", _dp), ("quats64", _dp), ("opac64", _dp), ("sh64", _dp),
        ("nv", C.c_int), ("wh", _i32p), ("intr", _fp), ("viewmats", _fp), ("viewmats64", _dp),
        ("campos64", _dp), ("subset_data", _u32p), ("subset_off", _i64p), ("counts", _i64p),
        ("tile_w", C.c_int), ("tile_h", C.c_int), ("near_plane", C.c_float), ("bg", C.c_double * 3),
        ("intr64", _dp),
    ]


class _Mirror(C.Structure):
    _fields_ = [("flags", _u32p), ("zbits", _u32p), ("radius", _i32p), ("rect", _i32p),
                ("tiles", _i32p), ("blend", _fp), ("colour", _fp), ("conic", _fp)]


class _Lists(C.Structure):
    _fields_ = [("vals", _u32p), ("ranges", _u32p), ("brute", C.c_int), ("decide64", C.c_int)]


class _Block(C.Structure):
    _fields_ = [("view", C.c_int), ("x0", C.c_int), ("y0", C.c_int), ("w", C.c_int), ("h", C.c_int)]


def _declare(L):
    L.orc_exp2_f32.argtypes = [C.c_float]; L.orc_exp2_f32.restype = C.c_float
    L.orc_exp_f32.argtypes = [C.c_float]; L.orc_exp_f32.restype = C.c_float
    L.orc_sh_basis_f32.argtypes = [C.c_int, C.c_float, C.c_float, C.c_float, _fp]
    L.orc_sh_basis_f64.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, _dp, _dp]
    L.orc_mirror_preprocess.argtypes = [C.POINTER(_Scene), C.POINTER(_Mirror)]
    L.orc_build_lists.argtypes = [C.POINTER(_Scene), C.POINTER(_Mirror), C.c_int64, _u64p, _u32p, _u32p]
    L.orc_count_instances.argtypes = [C.POINTER(_Scene), C.POINTER(_Mirror), C.POINTER(C.c_uint8)]
    L.orc_count_instances.restype = C.c_int64
    L.orc_build_lists_masked.argtypes = [C.POINTER(_Scene), C.POINTER(_Mirror), C.POINTER(C.c_uint8), C.c_int64,
                                         _u64p, _u32p, _u32p]
    L.orc_build_lists_masked.restype = C.c_int
    L.orc_preprocess64.argtypes = [C.POINTER(_Scene), C.POINTER(_Mirror), _dp]
    L.orc_rect64.argtypes = [C.POINTER(_Scene), C.POINTER(_Mirror), _i32p]
    L.orc_forward.argtypes = [C.POINTER(_Scene), C.POINTER(_Mirror), _dp, C.POINTER(_Lists),
                              C.POINTER(_Block), C.c_int, _dp, _dp, _dp, _dp, _u32p, _u32p, _u32p, _u32p]
    L.orc_tile_reach.argtypes = [C.POINTER(_Scene), C.POINTER(_Mirror), C.POINTER(_Lists), C.c_int64,
                                 C.POINTER(C.c_uint8)]
    L.orc_backward.argtypes = [C.POINTER(_Scene), C.POINTER(_Mirror), _dp, C.POINTER(_Lists),
                               C.POINTER(_Block), C.c_int, _dp, _dp, _dp,
                               _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_chain_backward.argtypes = [C.POINTER(_Scene), C.POINTER(_Mirror), _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                     _dp]
    L.orc_chain_backward.restype = C.c_int
    L.orc_num_threads.argtypes = []; L.orc_num_threads.restype = C.c_int
    L.orc_log_taps.argtypes = [C.c_double, C.POINTER(C.c_int), _fp, _dp]; L.orc_log_taps.restype = C.c_int
    L.orc_insertion.argtypes = [C.c_int, C.c_int, _fp, _fp, _fp, C.c_float, C.c_double, C.c_float,
                                _dp, _dp, _dp, _dp, C.POINTER(C.c_uint8)]
    L.orc_insertion.restype = C.c_int
    L.orc_set_num_threads.argtypes = [C.c_int]; L.orc_set_num_threads.restype = None
    for fn in ("orc_mirror_preprocess", "orc_build_lists", "orc_preprocess64", "orc_rect64",
               "orc_forward", "orc_backward", "orc_tile_reach"):
        getattr(L, fn).restype = C.c_int


def _ptr(a: Optional[np.ndarray], t):
    if a is None:
        return C.cast(None, t)
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(t)


# ----------------------------------------------------------------------------
# scalar helpers
# ----------------------------------------------------------------------------

def exp_f32(x: float) -> float:
    return float(lib().orc_exp_f32(float(x)))


def exp2_f32(x: float) -> float:
    return float(lib().orc_exp2_f32(float(x)))


def sh_basis_f32(degree: int, d) -> np.ndarray:
    out = np.zeros(16, dtype=np.float32)
    lib().orc_sh_basis_f32(degree, float(d[0]), float(d[1]), float(d[2]), _ptr(out, _fp))
    return out[: (degree + 1) ** 2]


def sh_basis_f64(degree: int, d) -> Tuple[np.ndarray, np.ndarray]:
    b = np.zeros(16, dtype=np.float64)
    db = np.zeros((16, 3), dtype=np.float64)
    lib().orc_sh_basis_f64(degree, float(d[0]), float(d[1]), float(d[2]), _ptr(b, _dp), _ptr(db, _dp))
    k = (degree + 1) ** 2
    return b[:k], db[:k]


# ----------------------------------------------------------------------------
# one oracle evaluation of a scene
# ----------------------------------------------------------------------------

class Oracle:
    """Oracle state for one scene: binary32 decisions, lists and FP64 values.

    ``params64`` (dict with means, log_scales, quats, opacity_logits, sh as
    float64) and ``viewmats64`` ([V,4,4] float64) replace the FP64 value-path
    inputs, e.g. for finite differences; the decision mirror always reads the
    binary32 scene, so decisions stay frozen under such perturbations.
    ``campos64`` ([V,3]) fixes the SH camera centre (the pose-detached path).
    """

    def __init__(self, scene, tile: Optional[Sequence[int]] = None, near: float = 0.2,
                 bg: Optional[Sequence[float]] = None):
        self.scene = scene
        self.tile = tuple(tile) if tile is not None else tuple(scene.tile)
        self.near = float(near)
        self.bg = tuple(bg) if bg is not None else tuple(scene.bg)
        s = scene
        f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
        self.means = f32(s.means); self.log_scales = f32(s.log_scales); self.quats = f32(s.quats)
        self.opac = f32(s.opacity_logits)
        self.sh = f32(s.sh.reshape(s.n, (s.sh_degree + 1) ** 2, 3))
        self.views = s.views
        nv = len(s.views)
        self.wh = np.array([[v.width, v.height] for v in s.views], dtype=np.int32)
        self.intr = np.array([[v.fx, v.fy, v.cx, v.cy] for v in s.views], dtype=np.float32)
        self.viewmats = np.ascontiguousarray(np.stack([np.asarray(v.viewmat, np.float32) for v in s.views]))
        subs, offs, counts, o = [], [], [], 0
        for v in s.views:
            if v.subset is None:
                offs.append(-1); counts.append(s.n)
            else:
                sub = np.ascontiguousarray(v.subset, dtype=np.uint32)
                subs.append(sub); offs.append(o); counts.append(sub.shape[0]); o += sub.shape[0]
        self.subset_data = np.ascontiguousarray(np.concatenate(subs)) if subs else np.zeros(1, np.uint32)
        self.subset_off = np.array(offs, dtype=np.int64)
        self.counts = np.array(counts, dtype=np.int64)
        self.rec_base = np.concatenate([[0], np.cumsum(self.counts)]).astype(np.int64)
        self.nvg = int(self.rec_base[-1])
        tx = [(v.width + self.tile[0] - 1) // self.tile[0] for v in s.views]
        ty = [(v.height + self.tile[1] - 1) // self.tile[1] for v in s.views]
        self.tiles_xy = list(zip(tx, ty))
        self.tile_base = np.concatenate([[0], np.cumsum([a * b for a, b in self.tiles_xy])]).astype(np.int64)
        self.n_tiles = int(self.tile_base[-1])
        self.set_values()
        self._m = None
        self._lists = None
        self._rec64 = None

    # -- value-path inputs ---------------------------------------------------
    def set_values(self, params64=None, viewmats64=None, campos64=None, intr64=None):
        s = self.scene
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        p = params64 or {}
        self.means64 = f64(p.get("means", s.means))
        self.log_scales64 = f64(p.get("log_scales", s.log_scales))
        self.quats64 = f64(p.get("quats", s.quats))
        self.opac64 = f64(p.get("opacity_logits", s.opacity_logits))
        self.sh64 = f64(p.get("sh", s.sh.reshape(s.n, (s.sh_degree + 1) ** 2, 3)))
        self.viewmats64 = f64(self.viewmats if viewmats64 is None else viewmats64)
        self.campos64 = None if campos64 is None else f64(campos64)
        # [V, 4] fx, fy, cx, cy for the value path (decisions keep the binary32 ones)
        self.intr64 = None if intr64 is None else f64(intr64)
        self._rec64 = None

    def _scene_struct(self) -> _Scene:
        st = _Scene()
        st.n = self.scene.n; st.sh_degree = self.scene.sh_degree
        st.means = _ptr(self.means, _fp); st.log_scales = _ptr(self.log_scales, _fp)
        st.quats = _ptr(self.quats, _fp); st.opac = _ptr(self.opac, _fp); st.sh = _ptr(self.sh, _fp)
        st.means64 = _ptr(self.means64, _dp); st.log_scales64 = _ptr(self.log_scales64, _dp)
        st.quats64 = _ptr(self.quats64, _dp); st.opac64 = _ptr(self.opac64, _dp); st.sh64 = _ptr(self.sh64, _dp)
        st.nv = len(self.views); st.wh = _ptr(self.wh, _i32p); st.intr = _ptr(self.intr, _fp)
        st.viewmats = _ptr(self.viewmats, _fp); st.viewmats64 = _ptr(self.viewmats64, _dp)
        st.campos64 = _ptr(self.campos64, _dp)
        st.subset_data = _ptr(self.subset_data, _u32p); st.subset_off = _ptr(self.subset_off, _i64p)
        st.counts = _ptr(self.counts, _i64p)
        st.tile_w, st.tile_h = self.tile
        st.near_plane = self.near
        st.bg = (C.c_double * 3)(*self.bg)
        st.intr64 = _ptr(getattr(self, "intr64", None), _dp)
        return st

    # -- decisions -------------------------------------------------------------
    def mirror(self) -> dict:
        if self._m is None:
            n = self.nvg
            m = dict(flags=np.zeros(n, np.uint32), zbits=np.zeros(n, np.uint32), radius=np.zeros(n, np.int32),
                     rect=np.zeros((n, 4), np.int32), tiles=np.zeros(n, np.int32),
                     blend=np.zeros((n, 6), np.float32), colour=np.zeros((n, 3), np.float32),
                     conic=np.zeros((n, 3), np.float32))
            self._m = m
            self._mst = _Mirror(_ptr(m["flags"], _u32p), _ptr(m["zbits"], _u32p), _ptr(m["radius"], _i32p),
                                _ptr(m["rect"], _i32p), _ptr(m["tiles"], _i32p), _ptr(m["blend"], _fp),
                                _ptr(m["colour"], _fp), _ptr(m["conic"], _fp))
            st = self._scene_struct()
            rc = lib().orc_mirror_preprocess(C.byref(st), C.byref(self._mst))
            assert rc == 0
        return self._m

    def restrict_tiles(self, tiles):
        """Build the lists for the given global tile ids only (for sampled
        checks of large batches); later ``lists()``/``forward()`` use them."""
        self.mirror()
        mask = np.zeros(max(self.n_tiles, 1), np.uint8)
        mask[np.asarray(list(tiles), np.int64)] = 1
        st = self._scene_struct()
        mp = mask.ctypes.data_as(C.POINTER(C.c_uint8))
        M = int(lib().orc_count_instances(C.byref(st), C.byref(self._mst), mp))
        keys = np.zeros(max(M, 1), np.uint64)
        vals = np.zeros(max(M, 1), np.uint32)
        ranges = np.zeros((max(self.n_tiles, 1), 2), np.uint32)
        rc = lib().orc_build_lists_masked(C.byref(st), C.byref(self._mst), mp, M, _ptr(keys, _u64p),
                                          _ptr(vals, _u32p), _ptr(ranges, _u32p))
        assert rc == 0, f"orc_build_lists_masked failed ({rc})"
        self._lists = (keys[:M], vals[:M], ranges[: self.n_tiles], vals)
        return self._lists[:3]

    def lists(self):
        """(keys u64[M], vals u32[M], ranges u32[n_tiles, 2]): every non-culled
        record in every tile of its rectangle, sorted by (tile, depth bits,
        record index)."""
        if self._lists is None:
            self.mirror()
            st = self._scene_struct()
            M = int(lib().orc_count_instances(C.byref(st), C.byref(self._mst), None))
            keys = np.zeros(max(M, 1), np.uint64)
            vals = np.zeros(max(M, 1), np.uint32)
            ranges = np.zeros((max(self.n_tiles, 1), 2), np.uint32)
            rc = lib().orc_build_lists(C.byref(st), C.byref(self._mst), M, _ptr(keys, _u64p),
                                       _ptr(vals, _u32p), _ptr(ranges, _u32p))
            assert rc == 0, f"orc_build_lists failed ({rc})"
            self._lists = (keys[:M], vals[:M], ranges[: self.n_tiles], vals)
        return self._lists[:3]

    def rec64(self) -> np.ndarray:
        if self._rec64 is None:
            self.mirror()
            out = np.zeros((max(self.nvg, 1), 10), np.float64)
            st = self._scene_struct()
            rc = lib().orc_preprocess64(C.byref(st), C.byref(self._mst), _ptr(out, _dp))
            assert rc == 0
            self._rec64 = out
        return self._rec64

    def rect64(self) -> np.ndarray:
        self.mirror()
        out = np.zeros((max(self.nvg, 1), 6), np.int32)
        st = self._scene_struct()
        lib().orc_rect64(C.byref(st), C.byref(self._mst), _ptr(out, _i32p))
        return out[: self.nvg]

    # -- rendering -------------------------------------------------------------
    def full_blocks(self) -> List[Tuple[int, int, int, int, int]]:
        return [(i, 0, 0, v.width, v.height) for i, v in enumerate(self.views)]

    def _lists_struct(self, brute: int, decide64: int) -> _Lists:
        if brute:
            dummy = np.zeros(2, np.uint32)
            self._dummy = dummy
            return _Lists(_ptr(dummy, _u32p), _ptr(dummy, _u32p), brute, decide64)
        _, _, ranges = self.lists()
        self._ranges_c = np.ascontiguousarray(ranges.reshape(-1) if ranges.size else np.zeros(2, np.uint32))
        return _Lists(_ptr(self._lists[3], _u32p), _ptr(self._ranges_c, _u32p), 0, decide64)

    @staticmethod
    def _blocks_struct(blocks):
        arr = (_Block * len(blocks))()
        for i, b in enumerate(blocks):
            arr[i] = _Block(*[int(x) for x in b])
        return arr

    def forward(self, blocks=None, brute: int = 0, decide64: int = 0) -> dict:
        """Render ``blocks`` = [(view, x0, y0, w, h)] (default: every full view).

        brute=1: per-pixel list from all records whose rectangle holds the
        pixel's tile (no keys or ranges); brute=2: from all records of the view.
        Returns per-block lists of arrays: rgb (3,h,w), depth, alpha, tfinal,
        ncontrib, nexam, nblend and stoprec (h,w); stoprec is the record at
        which the walk stopped (transmittance below 1e-4), or 0xFFFFFFFF.
        """
        blocks = self.full_blocks() if blocks is None else list(blocks)
        rec = self.rec64()
        npix = sum(b[3] * b[4] for b in blocks)
        rgb = np.zeros(3 * npix, np.float64); depth = np.zeros(npix, np.float64)
        alpha = np.zeros(npix, np.float64); tf = np.zeros(npix, np.float64)
        nc = np.zeros(npix, np.uint32); ne = np.zeros(npix, np.uint32); nbl = np.zeros(npix, np.uint32)
        sr = np.zeros(npix, np.uint32)
        st = self._scene_struct()
        ls = self._lists_struct(brute, decide64)
        bs = self._blocks_struct(blocks)
        rc = lib().orc_forward(C.byref(st), C.byref(self._mst), _ptr(rec, _dp), C.byref(ls), bs, len(blocks),
                               _ptr(rgb, _dp), _ptr(depth, _dp), _ptr(alpha, _dp), _ptr(tf, _dp),
                               _ptr(nc, _u32p), _ptr(ne, _u32p), _ptr(nbl, _u32p), _ptr(sr, _u32p))
        assert rc == 0
        return _split_blocks(blocks, rgb=rgb, depth=depth, alpha=alpha, tfinal=tf, ncontrib=nc, nexam=ne,
                             nblend=nbl, stoprec=sr)

    def reach(self) -> np.ndarray:
        """u8[M] over the current lists (full or restricted): 1 where the
        entry's record passes the blend's alpha test at some in-view pixel
        centre of its tile (brute force over the tile's pixels)."""
        keys, _, _ = self.lists()
        M = int(keys.size)
        out = np.zeros(max(M, 1), np.uint8)
        st = self._scene_struct()
        ls = self._lists_struct(0, 0)
        rc = lib().orc_tile_reach(C.byref(st), C.byref(self._mst), C.byref(ls), M,
                                  out.ctypes.data_as(C.POINTER(C.c_uint8)))
        assert rc == 0
        return out[:M]

    def backward(self, dl_rgb, dl_depth=None, dl_alpha=None, blocks=None, brute: int = 0,
                 want_grec: bool = False) -> dict:
        """Exact adjoint.  dl_*: per-block lists matching ``forward``'s layout."""
        blocks = self.full_blocks() if blocks is None else list(blocks)
        rec = self.rec64()
        cat = lambda xs: np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).reshape(-1) for x in xs]))
        drgb = cat(dl_rgb)
        ddep = None if dl_depth is None else cat(dl_depth)
        dalp = None if dl_alpha is None else cat(dl_alpha)
        n, K = self.scene.n, (self.scene.sh_degree + 1) ** 2
        g = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
                 opacity_logits=np.zeros(n), sh=np.zeros((n, K, 3)), pose=np.zeros((len(self.views), 6)),
                 focal=np.zeros((len(self.views), 2)))
        grec = np.zeros((max(self.nvg, 1), 10)) if want_grec else None
        st = self._scene_struct()
        ls = self._lists_struct(brute, 0)
        bs = self._blocks_struct(blocks)
        rc = lib().orc_backward(C.byref(st), C.byref(self._mst), _ptr(rec, _dp), C.byref(ls), bs, len(blocks),
                                _ptr(drgb, _dp), _ptr(ddep, _dp), _ptr(dalp, _dp),
                                _ptr(g["means"], _dp), _ptr(g["log_scales"], _dp), _ptr(g["quats"], _dp),
                                _ptr(g["opacity_logits"], _dp), _ptr(g["sh"], _dp), _ptr(g["pose"], _dp),
                                _ptr(grec, _dp), _ptr(g["focal"], _dp))
        assert rc == 0
        if want_grec:
            g["grec"] = grec[: self.nvg]
        return g


def chain_backward(o: "Oracle", grec: np.ndarray) -> dict:
    """Preprocess adjoint only, from per-record 2D gradients
    grec [N_vg][10] = du, dv, dc0, dc1, dc2, dsigma, dr, dg, db, dz."""
    o.mirror()
    grec = np.ascontiguousarray(grec, dtype=np.float64)
    n, K = o.scene.n, (o.scene.sh_degree + 1) ** 2
    g = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
             opacity_logits=np.zeros(n), sh=np.zeros((n, K, 3)), pose=np.zeros((len(o.views), 6)),
             focal=np.zeros((len(o.views), 2)))
    st = o._scene_struct()
    rc = lib().orc_chain_backward(C.byref(st), C.byref(o._mst), _ptr(grec, _dp), _ptr(g["means"], _dp),
                                  _ptr(g["log_scales"], _dp), _ptr(g["quats"], _dp), _ptr(g["opacity_logits"], _dp),
                                  _ptr(g["sh"], _dp), _ptr(g["pose"], _dp), _ptr(g["focal"], _dp))
    assert rc == 0
    return g


def _split_blocks(blocks, **arrs):
    out = {k: [] for k in arrs}
    off = 0
    for (_, _, _, w, h) in blocks:
        n = w * h
        for k, a in arrs.items():
            if k == "rgb":
                out[k].append(a[3 * off: 3 * off + 3 * n].reshape(3, h, w))
            else:
                out[k].append(a[off: off + n].reshape(h, w))
        off += n
    return out


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on."""
    lib().orc_set_num_threads(int(n))


# -- insertion probability and scale initialisation (Sec. 3.2, Eq. 4-6) -------

def log_taps(sigma: float = 1.0) -> Tuple[np.ndarray, np.ndarray]:
    """Zero-mean Laplacian-of-Gaussian taps [(2r+1)^2] as (binary32, double)."""
    r = C.c_int(0)
    t32 = np.zeros(15 * 15, np.float32)
    t64 = np.zeros(15 * 15, np.float64)
    rc = lib().orc_log_taps(float(sigma), C.byref(r), _ptr(t32, _fp), _ptr(t64, _dp))
    assert rc == 0, "sigma out of range"
    K = 2 * r.value + 1
    return t32[: K * K].reshape(K, K), t64[: K * K].reshape(K, K)


def insertion(gt: np.ndarray, rendered: np.ndarray, depth: np.ndarray, focal: float, sigma: float = 1.0,
              tau_a: float = 0.2) -> dict:
    """One view: gt, rendered [3, H, W] binary32, depth [H, W].  Returns the
    double-precision P(I), P(I~), P_a and S (0 where nothing is inserted) and
    the binary32 insertion decision P_a > tau_a."""
    gt = np.ascontiguousarray(gt, np.float32)
    rendered = np.ascontiguousarray(rendered, np.float32)
    depth = np.ascontiguousarray(depth, np.float32)
    _, H, W = gt.shape
    out = {k: np.zeros((H, W), np.float64) for k in ("p_gt", "p_ren", "p_a", "scale")}
    ins = np.zeros((H, W), np.uint8)
    rc = lib().orc_insertion(W, H, _ptr(gt, _fp), _ptr(rendered, _fp), _ptr(depth, _fp), float(focal), float(sigma),
                             float(tau_a), _ptr(out["p_gt"], _dp), _ptr(out["p_ren"], _dp), _ptr(out["p_a"], _dp),
                             _ptr(out["scale"], _dp), ins.ctypes.data_as(C.POINTER(C.c_uint8)))
    assert rc == 0, "orc_insertion failed"
    out["inserted"] = ins.astype(bool)
    return out


# -- rig chain (Sec. 3.1): V_i = A_i V_m --------------------------------------

def rig_chain(pose_grads, keyframe_of_view, rel, n_keyframes, focal_grads=None, camera_of_view=None,
              n_cameras=0) -> dict:
    """Gradients of a rig parametrisation from per-view ones.

    View i's world-to-camera pose is V_i = A_i V_m(k), A_i = [R_i | t_i] the
    fixed transform from the central camera m of keyframe k = keyframe_of_view[i]
    to camera i (the paper's T_i = T_m T_{i->m} for camera-to-world poses).  A
    left perturbation V_m <- exp(delta^) V_m reaches view i as
    Ad(A_i) delta, Ad(A) (rho, omega) = (R rho + t x (R omega), R omega), so
      dL/drho_m   = sum_i R_i^T g_rho_i
      dL/domega_m = sum_i R_i^T (g_omega_i - t_i x g_rho_i).
    The relative transform of rig camera c (Sec. 3.3 optimises those of the
    non-central cameras), perturbed on the left, A_c <- exp(delta^) A_c,
    perturbs each of its views' poses by the same delta:
    dL/ddelta_c = sum over views i of camera c of g_i.
    The focal length of rig camera c is shared by its views:
    dL/df_c = sum over views i of camera c of dL/df_i (fx and fy)."""
    g = np.asarray(pose_grads, np.float64).reshape(-1, 6)
    A = np.asarray(rel, np.float64).reshape(-1, 3, 4)
    kf = np.asarray(keyframe_of_view, np.int64)
    central = np.zeros((n_keyframes, 6))
    for i in range(g.shape[0]):
        R, t = A[i, :, :3], A[i, :, 3]
        gr, gw = g[i, :3], g[i, 3:]
        central[kf[i], :3] += R.T @ gr
        central[kf[i], 3:] += R.T @ (gw - np.cross(t, gr))
    out = {"central": central}
    if camera_of_view is not None:
        cam = np.asarray(camera_of_view, np.int64)
        cr = np.zeros((n_cameras, 6))
        for i in range(g.shape[0]):
            cr[cam[i]] += g[i]
        out["camera_rel"] = cr
    if focal_grads is not None:
        fg = np.asarray(focal_grads, np.float64).reshape(-1, 2)
        cam = np.asarray(camera_of_view, np.int64)
        cf = np.zeros((n_cameras, 2))
        for i in range(fg.shape[0]):
            cf[cam[i]] += fg[i]
        out["camera_focal"] = cf
    return out
