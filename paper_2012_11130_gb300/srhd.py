"""Python binding of libsrhd: the C-ABI entry points under the same names,
taking torch tensors (argument marshalling only; every step of the update
runs in the library's CUDA kernels).

Precision follows the tensor dtype: float64 -> SRHD_FP64, float32 ->
SRHD_MIXED (float storage; A of Eq. transcendental equation in double).
Every call also takes ``prec="mixed_cf"`` (float tensors) to select
SRHD_MIXED_CF, where A is formed by compensated float arithmetic and no
double arithmetic runs at all.
Layouts are those of include/srhd.h: SoA [5][n] for cell batches,
[npatch][5][12][12][12] ghosted patches, [npatch][5][8][8][8] interiors.

Tensors on the CPU are accepted by ``advance_patches`` and ``con2pri``: the
call then copies them to the device (pinned host memory makes the copies
asynchronous), runs there and copies the results back, which is the
end-to-end path a host-resident caller uses.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _native as N

__all__ = ["Params", "Context", "prim2con", "con2pri", "flux_patches", "advance_patches",
           "cfl_dt", "cfl_dt_noalloc", "fill_ghosts_uniform", "fill_ghosts_uniform3",
           "advance_patches_vl", "amr_fill_ghosts", "amr_restrict",
           "amr_flux_correct", "amr_prolong", "default_context"]


@dataclass
class Params:
    """Run-time parameters (Sections 3.1-3.3 of arXiv 2012.11130)."""
    cfl: float = 0.5
    theta: float = 1.5
    retry_factor: float = 0.75
    theta_floor: float = 1e-2
    riemann: str = "hllc"        # "hllc" | "hlle"
    cfl_mode: str = "signal"     # "signal" | "light"
    ndim: int = 3
    newton_max_iter: int = 0
    patch_variant: int = 0       # launch variant of the fused kernel (autotune.py)
    scheme: str = "reduced"      # "reduced" (Etilde, the paper's) | "total" (original, E)
    eos: str = "tm"              # "tm" (Taub-Mathews, the paper's) | "polytropic"
    gamma: float = 5.0 / 3.0     # Gamma of the polytropic EoS, 1 < gamma <= 5/3

    def to_c(self) -> N.Params:
        return N.Params(self.cfl, self.theta, self.retry_factor, self.theta_floor,
                        {"hllc": N.SRHD_HLLC, "hlle": N.SRHD_HLLE}[self.riemann],
                        {"signal": N.SRHD_CFL_SIGNAL, "light": N.SRHD_CFL_LIGHT}[self.cfl_mode],
                        self.ndim, self.newton_max_iter, self.patch_variant,
                        {"reduced": N.SRHD_SCHEME_REDUCED, "total": N.SRHD_SCHEME_TOTAL}[self.scheme],
                        {"tm": N.SRHD_EOS_TM, "polytropic": N.SRHD_EOS_POLYTROPIC}[self.eos],
                        self.gamma)


_PREC = {"fp64": (N.SRHD_FP64, torch.float64), "mixed": (N.SRHD_MIXED, torch.float32),
         "mixed_cf": (N.SRHD_MIXED_CF, torch.float32)}


def _prec(t: torch.Tensor, prec: str | None = None) -> int:
    if prec is not None:
        code, dt = _PREC[prec]
        if t.dtype != dt:
            raise TypeError(f"precision {prec!r} needs {dt} tensors, got {t.dtype}")
        return code
    if t.dtype == torch.float64:
        return N.SRHD_FP64
    if t.dtype == torch.float32:
        return N.SRHD_MIXED
    raise TypeError(f"unsupported dtype {t.dtype}: use float64 (FP64) or float32 (mixed)")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need_cuda(t: torch.Tensor, name: str, dtype=None):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")


class Context:
    """Owns an srhd_ctx* on one device (scratch for the CFL reduction)."""

    def __init__(self, params: Params | None = None, device: int | None = None):
        self._L = N.load()
        self.params = params or Params()
        self.device = torch.cuda.current_device() if device is None else device
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            p = self.params.to_c()
            N.check(self._L.srhd_create(ctypes.byref(self._h), ctypes.byref(p)), "srhd_create")

    def close(self):
        if self._h:
            self._L.srhd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- Section 2.3 ---------------------------------------------------------
    def prim2con(self, prim, cons=None, stream=None, prec=None):
        _need_cuda(prim, "prim")
        n = prim.shape[-1]
        if cons is None:
            cons = torch.empty_like(prim)
        _need_cuda(cons, "cons", prim.dtype)
        N.check(self._L.srhd_prim2con(self._h, _prec(prim, prec), _ptr(prim), _ptr(cons), n, n,
                                      _stream(stream)), "srhd_prim2con")
        return cons

    def con2pri(self, cons, prim=None, cell_status=None, stream=None, prec=None):
        host = not cons.is_cuda
        if host:
            dev = torch.device("cuda", self.device)
            cons_d = cons.to(dev, non_blocking=True)
        else:
            cons_d = cons
        _need_cuda(cons_d, "cons")
        n = cons_d.shape[-1]
        prim_d = torch.empty_like(cons_d) if (prim is None or host) else prim
        _need_cuda(prim_d, "prim", cons_d.dtype)
        st_d = cell_status
        if host and cell_status is not None:
            st_d = torch.empty(n, dtype=torch.int32, device=cons_d.device)
        if st_d is not None:
            _need_cuda(st_d, "cell_status", torch.int32)
        N.check(self._L.srhd_con2pri(self._h, _prec(cons_d, prec), _ptr(cons_d), _ptr(prim_d), n, n,
                                     _ptr(st_d), _stream(stream)), "srhd_con2pri")
        if host:
            out = prim if prim is not None else torch.empty(prim_d.shape, dtype=prim_d.dtype,
                                                            pin_memory=True)
            out.copy_(prim_d, non_blocking=True)
            if cell_status is not None:
                cell_status.copy_(st_d, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            return out
        return prim_d

    # ---- Section 3.1-3.3 -----------------------------------------------------
    def flux_patches(self, cons_ghosted, dt_dh, face_flux=None, patch_status=None, stream=None,
                     prec=None):
        _need_cuda(cons_ghosted, "cons_ghosted")
        npatch = cons_ghosted.shape[0]
        if face_flux is None:
            face_flux = torch.empty((npatch, 3, 5, 576), dtype=cons_ghosted.dtype,
                                    device=cons_ghosted.device)
        _need_cuda(face_flux, "face_flux", cons_ghosted.dtype)
        _need_cuda(dt_dh, "dt_dh", torch.float64)
        if patch_status is not None:
            _need_cuda(patch_status, "patch_status", torch.int32)
        N.check(self._L.srhd_flux_patches(self._h, _prec(cons_ghosted, prec), _ptr(cons_ghosted),
                                          _ptr(face_flux), npatch, _ptr(dt_dh), _ptr(patch_status),
                                          _stream(stream)), "srhd_flux_patches")
        return face_flux

    def advance_patches(self, cons_ghosted, dt_dh, cons_out=None, patch_face_flux=None,
                        worklist=None, dt_next=None, patch_status=None, npatch=None, stream=None,
                        prec=None):
        """One step of a batch of ghosted patches. Device tensors in, device
        tensors out; with a CPU ``cons_ghosted`` the call copies it in, runs
        and copies ``cons_out`` (and ``dt_next`` if given) back to the host."""
        if not cons_ghosted.is_cuda:
            return self._advance_host(cons_ghosted, dt_dh, cons_out, dt_next, patch_status, stream,
                                      prec)
        _need_cuda(cons_ghosted, "cons_ghosted")
        if npatch is None:
            npatch = worklist.numel() if worklist is not None else cons_ghosted.shape[0]
        if cons_out is None:
            cons_out = torch.empty((cons_ghosted.shape[0], 5, 8, 8, 8), dtype=cons_ghosted.dtype,
                                   device=cons_ghosted.device)
        _need_cuda(cons_out, "cons_out", cons_ghosted.dtype)
        _need_cuda(dt_dh, "dt_dh", torch.float64)
        for name, t, dt in (("patch_face_flux", patch_face_flux, cons_ghosted.dtype),
                            ("worklist", worklist, torch.int32), ("dt_next", dt_next, torch.float64),
                            ("patch_status", patch_status, torch.int32)):
            if t is not None:
                _need_cuda(t, name, dt)
        N.check(self._L.srhd_advance_patches(
            self._h, _prec(cons_ghosted, prec), _ptr(cons_ghosted), _ptr(cons_out),
            _ptr(patch_face_flux), npatch, _ptr(dt_dh), _ptr(worklist), _ptr(dt_next),
            _ptr(patch_status), _stream(stream)), "srhd_advance_patches")
        return cons_out

    def _advance_host(self, cons_ghosted, dt_dh, cons_out, dt_next, patch_status, stream, prec,
                      chunks: int = 8):
        """Host-resident batch: the batch is cut into chunks whose
        host-to-device copy, fused step and device-to-host copy run on three
        streams, so copies of one chunk overlap the step of another (pinned
        host tensors make the copies asynchronous). The per-chunk CFL minima
        are combined at the end. Device buffers are kept for reuse."""
        dev = torch.device("cuda", self.device)
        n = cons_ghosted.shape[0]
        dtype = cons_ghosted.dtype
        key = (n, dtype)
        if getattr(self, "_host_buf_key", None) != key:
            self._host_buf = dict(
                g=torch.empty((n, 5, 12, 12, 12), dtype=dtype, device=dev),
                dd=torch.empty((n, 2), dtype=torch.float64, device=dev),
                out=torch.empty((n, 5, 8, 8, 8), dtype=dtype, device=dev),
                st=torch.empty(n, dtype=torch.int32, device=dev),
                wl=torch.arange(n, dtype=torch.int32, device=dev),
                dn=torch.empty(chunks, dtype=torch.float64, device=dev),
                streams=[torch.cuda.Stream(device=dev) for _ in range(3)])
            self._host_buf_key = key
        b = self._host_buf
        h2d, comp, d2h = b["streams"]
        if cons_out is None:
            cons_out = torch.empty((n, 5, 8, 8, 8), dtype=dtype, pin_memory=True)
        cur = stream or torch.cuda.current_stream(dev)
        h2d.wait_stream(cur)
        comp.wait_stream(cur)
        d2h.wait_stream(cur)
        bounds = [n * k // chunks for k in range(chunks + 1)]
        used = 0
        for k in range(chunks):
            a, e = bounds[k], bounds[k + 1]
            if a == e:
                continue
            used = k + 1
            with torch.cuda.stream(h2d):
                b["g"][a:e].copy_(cons_ghosted[a:e], non_blocking=True)
                b["dd"][a:e].copy_(dt_dh[a:e], non_blocking=True)
            comp.wait_stream(h2d)
            self.advance_patches(b["g"], b["dd"], cons_out=b["out"], worklist=b["wl"][a:e],
                                 npatch=e - a, dt_next=b["dn"][k:k + 1] if dt_next is not None
                                 else None, patch_status=b["st"], stream=comp, prec=prec)
            d2h.wait_stream(comp)
            with torch.cuda.stream(d2h):
                cons_out[a:e].copy_(b["out"][a:e], non_blocking=True)
                if patch_status is not None:
                    patch_status[a:e].copy_(b["st"][a:e], non_blocking=True)
        d2h.synchronize()
        if dt_next is not None:
            dn = b["dn"][:used].cpu()
            dt_next.copy_(dn.min().reshape(1) if not torch.isnan(dn).any()
                          else torch.full((1,), float("nan"), dtype=torch.float64))
        return cons_out

    def cfl_dt(self, cons, dh, dt_out=None, stream=None, prec=None):
        _need_cuda(cons, "cons")
        if dt_out is None:
            dt_out = torch.empty(1, dtype=torch.float64, device=cons.device)
        _need_cuda(dt_out, "dt_out", torch.float64)
        N.check(self._L.srhd_cfl_dt(self._h, _prec(cons, prec), _ptr(cons), cons.shape[0], float(dh),
                                    _ptr(dt_out), _stream(stream)), "srhd_cfl_dt")
        return dt_out

    def fill_ghosts_uniform(self, interior, npx, npy, npz, bc=("periodic",) * 3, ghosted=None,
                            stream=None):
        _need_cuda(interior, "interior")
        if ghosted is None:
            ghosted = torch.empty((interior.shape[0], 5, 12, 12, 12), dtype=interior.dtype,
                                  device=interior.device)
        _need_cuda(ghosted, "ghosted", interior.dtype)
        code = {"periodic": N.SRHD_BC_PERIODIC, "outflow": N.SRHD_BC_OUTFLOW}
        bcs = (ctypes.c_int32 * 3)(*[code[b] for b in bc])
        N.check(self._L.srhd_fill_ghosts_uniform(self._h, _prec(interior), _ptr(interior),
                                                 _ptr(ghosted), npx, npy, npz, bcs,
                                                 _stream(stream)), "srhd_fill_ghosts_uniform")
        return ghosted

    def advance_uniform(self, interior, npx, npy, npz, dt_dh, bc=("periodic",) * 3, p0=0,
                        n=None, cons_out=None, patch_face_flux=None, dt_next=None,
                        patch_status=None, stream=None, prec=None):
        """One fused step of patches p0 .. p0+n-1 of a device-resident
        uniform grid (srhd_advance_uniform): the ghost zones are read from
        the neighbouring patches of `interior` [np][5][8][8][8] (patch
        (ix, iy, iz) at (iz*npy + iy)*npx + ix); no ghosted copy is made.
        Returns cons_out [n][5][8][8][8]."""
        _need_cuda(interior, "interior")
        npatch = npx * npy * npz
        if n is None:
            n = npatch - p0
        if interior.shape[0] != npatch:
            raise ValueError(f"interior holds {interior.shape[0]} patches, grid has {npatch}")
        if cons_out is None:
            cons_out = torch.empty((n, 5, 8, 8, 8), dtype=interior.dtype, device=interior.device)
        _need_cuda(cons_out, "cons_out", interior.dtype)
        _need_cuda(dt_dh, "dt_dh", torch.float64)
        for name, t, dt in (("patch_face_flux", patch_face_flux, interior.dtype),
                            ("dt_next", dt_next, torch.float64),
                            ("patch_status", patch_status, torch.int32)):
            if t is not None:
                _need_cuda(t, name, dt)
        code = {"periodic": N.SRHD_BC_PERIODIC, "outflow": N.SRHD_BC_OUTFLOW}
        bcs = (ctypes.c_int32 * 3)(*[code[b] for b in bc])
        N.check(self._L.srhd_advance_uniform(
            self._h, _prec(interior, prec), _ptr(interior), npx, npy, npz, bcs, p0, n,
            _ptr(cons_out), _ptr(patch_face_flux), _ptr(dt_dh), _ptr(dt_next),
            _ptr(patch_status), _stream(stream)), "srhd_advance_uniform")
        return cons_out

    def con2pri_patches(self, cons, prim_out=None, stream=None, prec=None):
        """Primitive cache of interior patches (srhd_con2pri_patches):
        cons [np][5][8][8][8] -> [np][6][8][8][8] = (rho, U^x, U^y, U^z, p,
        tau), NaN for unphysical cells."""
        _need_cuda(cons, "cons")
        n = cons.shape[0]
        if prim_out is None:
            prim_out = torch.empty((n, 6, 8, 8, 8), dtype=cons.dtype, device=cons.device)
        _need_cuda(prim_out, "prim_out", cons.dtype)
        N.check(self._L.srhd_con2pri_patches(self._h, _prec(cons, prec), _ptr(cons), n,
                                             _ptr(prim_out), _stream(stream)),
                "srhd_con2pri_patches")
        return prim_out

    def advance_uniform_prim(self, interior, prim_in, npx, npy, npz, dt_dh, bc=("periodic",) * 3,
                             p0=0, n=None, cons_out=None, prim_out=None, patch_face_flux=None,
                             dt_next=None, patch_status=None, stream=None, prec=None):
        """advance_uniform with the primitive cache (srhd_advance_uniform_prim):
        the tiles' primitives come from prim_in [np][6][8][8][8] (from
        con2pri_patches or the previous step's prim_out) and the new state's
        are written to prim_out. Returns (cons_out, prim_out)."""
        _need_cuda(interior, "interior")
        _need_cuda(prim_in, "prim_in", interior.dtype)
        npatch = npx * npy * npz
        if n is None:
            n = npatch - p0
        if interior.shape[0] != npatch or prim_in.shape[0] != npatch:
            raise ValueError(f"interior/prim_in must hold the grid's {npatch} patches")
        if cons_out is None:
            cons_out = torch.empty((n, 5, 8, 8, 8), dtype=interior.dtype, device=interior.device)
        if prim_out is None:
            prim_out = torch.empty((n, 6, 8, 8, 8), dtype=interior.dtype, device=interior.device)
        _need_cuda(cons_out, "cons_out", interior.dtype)
        _need_cuda(prim_out, "prim_out", interior.dtype)
        _need_cuda(dt_dh, "dt_dh", torch.float64)
        for name, t, dt in (("patch_face_flux", patch_face_flux, interior.dtype),
                            ("dt_next", dt_next, torch.float64),
                            ("patch_status", patch_status, torch.int32)):
            if t is not None:
                _need_cuda(t, name, dt)
        code = {"periodic": N.SRHD_BC_PERIODIC, "outflow": N.SRHD_BC_OUTFLOW}
        bcs = (ctypes.c_int32 * 3)(*[code[b] for b in bc])
        N.check(self._L.srhd_advance_uniform_prim(
            self._h, _prec(interior, prec), _ptr(interior), _ptr(prim_in), npx, npy, npz, bcs, p0,
            n, _ptr(cons_out), _ptr(prim_out), _ptr(patch_face_flux), _ptr(dt_dh), _ptr(dt_next),
            _ptr(patch_status), _stream(stream)), "srhd_advance_uniform_prim")
        return cons_out, prim_out

    def advance_uniform_host(self, interior, npx, npy, npz, dt, dh, bc=("periodic",) * 3,
                             cons_out=None, patch_status=None, chunks=32, stream=None, prec=None):
        """One step of a uniform grid held in host memory
        (srhd_advance_uniform_host): interior [np][5][8][8][8] CPU tensor
        (pinned for overlapped copies), patch (ix, iy, iz) at index
        (iz*npy + iy)*npx + ix. Returns (cons_out, dt_next); cons_out may be
        `interior` itself."""
        if interior.device.type != "cpu" or not interior.is_contiguous():
            raise ValueError("interior must be a contiguous host tensor")
        n = npx * npy * npz
        if tuple(interior.shape) != (n, 5, 8, 8, 8):
            raise ValueError(f"interior must be [{n}][5][8][8][8], got {tuple(interior.shape)}")
        if cons_out is None:
            cons_out = torch.empty_like(interior, pin_memory=interior.is_pinned())
        if (cons_out.device.type != "cpu" or cons_out.dtype != interior.dtype
                or cons_out.shape != interior.shape or not cons_out.is_contiguous()):
            raise ValueError("cons_out must be a contiguous host tensor like interior")
        if patch_status is not None and (patch_status.device.type != "cpu"
                                         or patch_status.dtype != torch.int32
                                         or patch_status.numel() < n):
            raise ValueError("patch_status must be a host int32 tensor of npatch entries")
        code = {"periodic": N.SRHD_BC_PERIODIC, "outflow": N.SRHD_BC_OUTFLOW}
        bcs = (ctypes.c_int32 * 3)(*[code[b] for b in bc])
        dn = ctypes.c_double(0.0)
        st = (ctypes.cast(patch_status.data_ptr(), ctypes.POINTER(ctypes.c_int32))
              if patch_status is not None else None)
        N.check(self._L.srhd_advance_uniform_host(
            self._h, _prec(interior, prec), _ptr(interior), _ptr(cons_out), npx, npy, npz, bcs,
            float(dt), float(dh), ctypes.byref(dn), st, int(chunks), _stream(stream)),
            "srhd_advance_uniform_host")
        return cons_out, dn.value

    # ---- VL integrator (include/srhd.h: srhd_advance_patches_vl) ---------------
    def advance_patches_vl(self, cons_ghosted, dt_dh, cons_out=None, patch_face_flux=None,
                           worklist=None, dt_next=None, patch_status=None, npatch=None,
                           stream=None, prec=None):
        """One VL step of device patches with three ghost cells,
        [npatch][5][14][14][14] -> [npatch][5][8][8][8]."""
        _need_cuda(cons_ghosted, "cons_ghosted")
        if npatch is None:
            npatch = worklist.numel() if worklist is not None else cons_ghosted.shape[0]
        if cons_out is None:
            cons_out = torch.empty((cons_ghosted.shape[0], 5, 8, 8, 8), dtype=cons_ghosted.dtype,
                                   device=cons_ghosted.device)
        _need_cuda(cons_out, "cons_out", cons_ghosted.dtype)
        _need_cuda(dt_dh, "dt_dh", torch.float64)
        for name, t, dt in (("patch_face_flux", patch_face_flux, cons_ghosted.dtype),
                            ("worklist", worklist, torch.int32), ("dt_next", dt_next, torch.float64),
                            ("patch_status", patch_status, torch.int32)):
            if t is not None:
                _need_cuda(t, name, dt)
        N.check(self._L.srhd_advance_patches_vl(
            self._h, _prec(cons_ghosted, prec), _ptr(cons_ghosted), _ptr(cons_out),
            _ptr(patch_face_flux), npatch, _ptr(dt_dh), _ptr(worklist), _ptr(dt_next),
            _ptr(patch_status), _stream(stream)), "srhd_advance_patches_vl")
        return cons_out

    def fill_ghosts_uniform3(self, interior, npx, npy, npz, bc=("periodic",) * 3, ghosted=None,
                             stream=None):
        """Uniform-grid ghost fill with three ghost cells ([np][5][14^3])."""
        _need_cuda(interior, "interior")
        if ghosted is None:
            ghosted = torch.empty((interior.shape[0], 5, 14, 14, 14), dtype=interior.dtype,
                                  device=interior.device)
        _need_cuda(ghosted, "ghosted", interior.dtype)
        code = {"periodic": N.SRHD_BC_PERIODIC, "outflow": N.SRHD_BC_OUTFLOW}
        bcs = (ctypes.c_int32 * 3)(*[code[b] for b in bc])
        N.check(self._L.srhd_fill_ghosts_uniform3(self._h, _prec(interior), _ptr(interior),
                                                  _ptr(ghosted), npx, npy, npz, bcs,
                                                  _stream(stream)), "srhd_fill_ghosts_uniform3")
        return ghosted

    # ---- AMR (include/srhd.h: srhd_amr_*) -------------------------------------
    def amr_fill_ghosts(self, cur, prev, ghosted, amr_map, p0, n, w=0.0, special=None,
                        stream=None, prec=None):
        """Ghost-zone fill of patches p0..p0+n-1 from the source map
        [ntotal][12^3] (int32); cur/prev [ntotal][5][8][8][8]."""
        _need_cuda(cur, "cur")
        _need_cuda(prev, "prev", cur.dtype)
        _need_cuda(ghosted, "ghosted", cur.dtype)
        _need_cuda(amr_map, "map", torch.int32)
        nsp = 0 if special is None else special.shape[0]
        if special is not None:
            _need_cuda(special, "special", cur.dtype)
        N.check(self._L.srhd_amr_fill_ghosts(self._h, _prec(cur, prec), _ptr(cur), _ptr(prev),
                                             _ptr(ghosted), _ptr(amr_map), cur.shape[0], p0, n,
                                             float(w), _ptr(special), nsp, _stream(stream)),
                "srhd_amr_fill_ghosts")
        return ghosted

    def advance_amr(self, level_state, coarse_old, coarse_new, amr_map, dt_dh, cons_out,
                    w=0.0, special=None, patch_face_flux=None, worklist=None, npatch=None,
                    dt_next=None, patch_status=None, stream=None, prec=None):
        """Ghost fill from the source map and fused step in one launch
        (srhd_advance_amr): map entries without the coarse bit read
        level_state, coarse ones (1-w) coarse_old + w coarse_new; the
        processed patches' rows of cons_out are written. All state arrays
        [ntotal][5][8][8][8]."""
        _need_cuda(level_state, "level_state")
        dt = level_state.dtype
        for name, t in (("coarse_old", coarse_old), ("coarse_new", coarse_new),
                        ("cons_out", cons_out)):
            _need_cuda(t, name, dt)
        _need_cuda(amr_map, "map", torch.int32)
        _need_cuda(dt_dh, "dt_dh", torch.float64)
        ntotal = level_state.shape[0]
        if npatch is None:
            npatch = worklist.numel() if worklist is not None else ntotal
        for name, t, tdt in (("patch_face_flux", patch_face_flux, dt),
                             ("worklist", worklist, torch.int32),
                             ("dt_next", dt_next, torch.float64),
                             ("patch_status", patch_status, torch.int32)):
            if t is not None:
                _need_cuda(t, name, tdt)
        nsp = 0 if special is None else special.shape[0]
        if special is not None:
            _need_cuda(special, "special", dt)
        N.check(self._L.srhd_advance_amr(
            self._h, _prec(level_state, prec), _ptr(level_state), _ptr(coarse_old),
            _ptr(coarse_new), _ptr(amr_map), ntotal, float(w), _ptr(special), nsp, _ptr(cons_out),
            _ptr(patch_face_flux), npatch, _ptr(dt_dh), _ptr(worklist), _ptr(dt_next),
            _ptr(patch_status), _stream(stream)), "srhd_advance_amr")
        return cons_out

    def amr_restrict(self, cur, children, stream=None, prec=None):
        """Fine -> coarse averaging; children [nparent][9] int32."""
        _need_cuda(cur, "cur")
        _need_cuda(children, "children", torch.int32)
        N.check(self._L.srhd_amr_restrict(self._h, _prec(cur, prec), _ptr(cur), _ptr(children),
                                          children.shape[0], cur.shape[0], _stream(stream)),
                "srhd_amr_restrict")
        return cur

    def amr_flux_correct(self, cur, flux_coarse, flux_fine0, flux_fine1, faces, dt_dh,
                         stream=None, prec=None, skipped=None):
        """Coarse-fine flux correction; faces [nrows][25] int32; patch-face
        fluxes [ntotal][6][5][64]; dt_dh [ntotal][2] float64; skipped
        (optional) one device int32 to which the number of cells whose
        correction was skipped (left unphysical by it) is added."""
        _need_cuda(cur, "cur")
        if skipped is not None:
            _need_cuda(skipped, "skipped", torch.int32)
        for t, nm in ((flux_coarse, "flux_coarse"), (flux_fine0, "flux_fine0"),
                      (flux_fine1, "flux_fine1")):
            _need_cuda(t, nm, cur.dtype)
        _need_cuda(faces, "faces", torch.int32)
        _need_cuda(dt_dh, "dt_dh", torch.float64)
        N.check(self._L.srhd_amr_flux_correct(self._h, _prec(cur, prec), _ptr(cur),
                                              _ptr(flux_coarse), _ptr(flux_fine0),
                                              _ptr(flux_fine1), _ptr(faces), faces.shape[0],
                                              _ptr(dt_dh), cur.shape[0], _ptr(skipped),
                                              _stream(stream)),
                "srhd_amr_flux_correct")
        return cur

    def amr_prolong(self, cur, prev, table, out, w=0.0, fallbacks=None, stream=None, prec=None):
        """Limited linear prolongation of coarse-sourced ghost cells (rows of
        `table` [nrows][8] int32) into `out` [nrows][5]; fallbacks (optional)
        one device int32 counting the rows interpolated in primitive
        variables."""
        _need_cuda(cur, "cur")
        _need_cuda(prev, "prev", cur.dtype)
        _need_cuda(out, "out", cur.dtype)
        _need_cuda(table, "table", torch.int32)
        if fallbacks is not None:
            _need_cuda(fallbacks, "fallbacks", torch.int32)
        if out.shape[0] < table.shape[0] or not out.is_contiguous():
            raise ValueError("out must be a contiguous [>= nrows][5] tensor")
        N.check(self._L.srhd_amr_prolong(self._h, _prec(cur, prec), _ptr(cur), _ptr(prev),
                                         _ptr(table), table.shape[0], cur.shape[0], float(w),
                                         _ptr(out), _ptr(fallbacks), _stream(stream)),
                "srhd_amr_prolong")
        return out


_default = {}


def default_context(params: Params | None = None) -> Context:
    dev = torch.cuda.current_device()
    key = (dev, None if params is None else tuple(vars(params).items()))
    if key not in _default:
        _default[key] = Context(params, dev)
    return _default[key]


def prim2con(prim, cons=None, stream=None, prec=None):
    return default_context().prim2con(prim, cons, stream, prec)


def con2pri(cons, prim=None, cell_status=None, stream=None, prec=None):
    return default_context().con2pri(cons, prim, cell_status, stream, prec)


def flux_patches(cons_ghosted, dt_dh, face_flux=None, patch_status=None, stream=None, prec=None):
    return default_context().flux_patches(cons_ghosted, dt_dh, face_flux, patch_status, stream,
                                          prec)


def advance_patches(cons_ghosted, dt_dh, **kw):
    return default_context().advance_patches(cons_ghosted, dt_dh, **kw)


def cfl_dt(cons, dh, dt_out=None, stream=None, prec=None):
    return default_context().cfl_dt(cons, dh, dt_out, stream, prec)


def cfl_dt_noalloc(cons, dh, dt_out=None, params: Params | None = None, stream=None, prec=None):
    """srhd_cfl_dt_noalloc: the CFL bound of interior patches [np][5][8][8][8]
    without a context (no device allocation by the library)."""
    _need_cuda(cons, "cons")
    if dt_out is None:
        dt_out = torch.empty(1, dtype=torch.float64, device=cons.device)
    _need_cuda(dt_out, "dt_out", torch.float64)
    L = N.load()
    p = (params or Params()).to_c()
    N.check(L.srhd_cfl_dt_noalloc(_prec(cons, prec), _ptr(cons), cons.shape[0], float(dh),
                                  ctypes.byref(p), _ptr(dt_out), _stream(stream)),
            "srhd_cfl_dt_noalloc")
    return dt_out


def fill_ghosts_uniform(interior, npx, npy, npz, bc=("periodic",) * 3, ghosted=None, stream=None):
    return default_context().fill_ghosts_uniform(interior, npx, npy, npz, bc, ghosted, stream)


def amr_fill_ghosts(cur, prev, ghosted, amr_map, p0, n, w=0.0, special=None, stream=None,
                    prec=None):
    return default_context().amr_fill_ghosts(cur, prev, ghosted, amr_map, p0, n, w, special,
                                             stream, prec)


def amr_restrict(cur, children, stream=None, prec=None):
    return default_context().amr_restrict(cur, children, stream, prec)


def amr_flux_correct(cur, flux_coarse, flux_fine0, flux_fine1, faces, dt_dh, stream=None,
                     prec=None, skipped=None):
    return default_context().amr_flux_correct(cur, flux_coarse, flux_fine0, flux_fine1, faces,
                                              dt_dh, stream, prec, skipped)


def amr_prolong(cur, prev, table, out, w=0.0, fallbacks=None, stream=None, prec=None):
    return default_context().amr_prolong(cur, prev, table, out, w, fallbacks, stream, prec)


def advance_patches_vl(cons_ghosted, dt_dh, **kw):
    return default_context().advance_patches_vl(cons_ghosted, dt_dh, **kw)


def fill_ghosts_uniform3(interior, npx, npy, npz, bc=("periodic",) * 3, ghosted=None,
                         stream=None):
    return default_context().fill_ghosts_uniform3(interior, npx, npy, npz, bc, ghosted, stream)
