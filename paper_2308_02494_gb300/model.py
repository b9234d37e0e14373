"""Tensor-owning wrapper over the libsrn C ABI.

``SRN`` allocates, with PyTorch, every device buffer the library needs (flat
parameter / gradient / Adam buffers laid out by ``srn_param_layout``, the BF16
shadow, the per-brick data range and the workspace), packs per-brick parameter
dicts into the flat layout, and forwards calls to the entry points of
``paper_2308_02494_gb300.srn``.  ``APMGSRNFunction`` puts the hand-written
adjoint (``srn_backward`` with ``SRN_UPSTREAM``) behind ``torch.autograd``.
All arithmetic runs in libsrn's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import srn as _s
from .synth import ModelShape


def _stream_ptr(stream) -> int:
    return (stream if stream is not None else torch.cuda.current_stream()).cuda_stream


class TiledVolume:
    """A volume in the tiled layout of srn_tile_volume (4^3-voxel tiles) for the ground-truth
    lookup; `dims` are the (x, y, z) extents of the volume it was made from."""

    def __init__(self, volume: torch.Tensor, stream=None):
        if volume.dim() != 3 or volume.dtype != torch.float32 or not volume.is_contiguous():
            raise ValueError("volume must be a contiguous float32 [z][y][x] tensor")
        self.dims = [volume.shape[2], volume.shape[1], volume.shape[0]]
        n = _s.srn_tiled_volume_bytes(self.dims) // 4
        self.data = torch.empty(n, dtype=torch.float32, device=volume.device)
        _s.srn_tile_volume(_stream_ptr(stream), volume.data_ptr(), self.dims, self.data.data_ptr())


class SRN:
    def __init__(self, shape: ModelShape, n_bricks: int = 1, precision: str = "fp32",
                 max_points: int = 1 << 18, device="cuda", flat_top_p: int = 10,
                 density_eps: float = 1e-8, lr_feat: float = 1e-2, lr_xform: float = 1e-3,
                 beta1: float = 0.9, beta2: float = 0.99, adam_eps: float = 1e-8):
        self.shape = shape
        self.n_bricks = n_bricks
        self.device = torch.device(device)
        self.bf16 = precision == "bf16"
        self.cfg = _s.Config(n_bricks, shape.n_grids, shape.channels, shape.res, shape.hidden,
                             _s.SRN_BF16 if self.bf16 else _s.SRN_FP32, flat_top_p, density_eps,
                             lr_feat, lr_xform, beta1, beta2, adam_eps)
        self.lay = _s.srn_param_layout(self.cfg)
        n, na = self.lay.n_params, self.lay.n_group_a
        kw = dict(device=self.device)
        self.params = torch.zeros(n, dtype=torch.float32, **kw)
        self.grads = torch.zeros(n, dtype=torch.float32, **kw)
        self.adam_m = torch.zeros(n, dtype=torch.float32, **kw)
        self.adam_v = torch.zeros(n, dtype=torch.float32, **kw)
        self.shadow = torch.zeros(na, dtype=torch.int16, **kw) if self.bf16 else None
        self.range = torch.zeros((n_bricks, 2), dtype=torch.float32, **kw)
        self.range[:, 1] = 1.0
        self.max_points = max_points
        wsb = _s.srn_workspace_size(self.cfg, max_points)
        self.workspace = torch.zeros(wsb + 256, dtype=torch.uint8, **kw)
        ws_ptr = (self.workspace.data_ptr() + 255) // 256 * 256
        t = _s.Tensors(self.params.data_ptr(), self.grads.data_ptr(), self.adam_m.data_ptr(),
                       self.adam_v.data_ptr(), self.shadow.data_ptr() if self.bf16 else None,
                       self.range.data_ptr())
        self.handle = _s.srn_create(self.cfg, t, ws_ptr, wsb, max_points)
        self.losses = torch.zeros((n_bricks, 4), dtype=torch.float64, **kw)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                _s.srn_destroy(h)
            except Exception:
                pass
            self.handle = None

    # ------------------------------------------------------------------ packing
    def _views(self, flat: torch.Tensor, b: int) -> dict:
        L, s = self.lay, self.shape
        M, R, C, H, K = s.n_grids, s.res, s.channels, s.hidden, s.feat
        return {
            "F": flat[L.off_F + b * L.size_F: L.off_F + b * L.size_F + M * R ** 3 * C].view(M, R, R, R, C),
            "W1": flat[L.off_W1 + b * L.size_W1: L.off_W1 + b * L.size_W1 + H * K].view(H, K),
            "W2": flat[L.off_W2 + b * L.size_W2: L.off_W2 + b * L.size_W2 + H * H].view(H, H),
            "w3": flat[L.off_w3 + b * L.size_w3: L.off_w3 + b * L.size_w3 + H],
            "G": flat[L.off_G + b * L.size_G: L.off_G + b * L.size_G + M * 12].view(M, 3, 4),
        }

    def pack(self, models) -> torch.Tensor:
        """A new flat float32 parameter tensor (the library's layout) holding one dict
        per brick (F, G, W1, W2, w3 as numpy arrays); padding entries are zero."""
        if isinstance(models, dict):
            models = [models]
        assert len(models) == self.n_bricks
        flat = torch.zeros_like(self.params)
        for b, m in enumerate(models):
            v = self._views(flat, b)
            for k in ("F", "W1", "W2", "w3", "G"):
                v[k].copy_(torch.as_tensor(np.asarray(m[k], dtype=np.float32)))
        return flat

    def set_params(self, models, stream=None) -> None:
        """models: one dict per brick (F, G, W1, W2, w3, vmin, vmax) of numpy arrays."""
        if isinstance(models, dict):
            models = [models]
        self.params.copy_(self.pack(models))
        for b, m in enumerate(models):
            self.range[b, 0] = float(m["vmin"])
            self.range[b, 1] = float(m["vmax"])
        self.adam_m.zero_()
        self.adam_v.zero_()
        self.sync_shadow(stream)

    def sync_shadow(self, stream=None) -> None:
        """Re-derive the BF16 shadow from the float32 parameters (srn_sync_shadow)."""
        _s.srn_sync_shadow(self.handle, _stream_ptr(stream))

    def get(self, which: str = "params") -> list:
        flat = {"params": self.params, "grads": self.grads, "m": self.adam_m, "v": self.adam_v}[which]
        out = []
        for b in range(self.n_bricks):
            d = {k: t.detach().cpu().numpy().astype(np.float64) for k, t in self._views(flat, b).items()}
            d["vmin"], d["vmax"] = float(self.range[b, 0]), float(self.range[b, 1])
            out.append(d)
        return out

    # ------------------------------------------------------------------ entry points
    @staticmethod
    def offsets_of(counts) -> list:
        return [0] + list(np.cumsum([int(c) for c in counts]))

    def forward(self, xyz: torch.Tensor, offsets, out: torch.Tensor | None = None, stream=None):
        if out is None:
            out = torch.empty(xyz.shape[0], dtype=torch.float32, device=self.device)
        _s.srn_forward(self.handle, _stream_ptr(stream), xyz.data_ptr(), offsets, out.data_ptr())
        return out

    def backward(self, xyz, target, offsets, density: bool = False, upstream: bool = False,
                 rec_dg: bool = False, stream=None):
        """srn_backward; rec_dg adds the gradient of L_rec (or of the upstream loss) into
        G through the features (SRN_REC_DG), which training leaves out."""
        flags = ((_s.SRN_DENSITY if density else 0) | (_s.SRN_UPSTREAM if upstream else 0)
                 | (_s.SRN_REC_DG if rec_dg else 0))
        _s.srn_backward(self.handle, _stream_ptr(stream), xyz.data_ptr(), target.data_ptr(), offsets,
                        flags, self.losses.data_ptr())
        return self.losses

    @property
    def tuning(self) -> dict:
        """Launch shape of the BF16 training pass (srn_get_tuning)."""
        return _s.srn_get_tuning(self.handle)

    def set_tuning(self, tile_points: int, tile_level: int, density_ctas: int) -> None:
        _s.srn_set_tuning(self.handle, tile_points, tile_level, density_ctas)

    def autotune(self, xyz, target, offsets, density: bool = True, reps: int = 5, stream=None) -> dict:
        """srn_autotune on one batch: times the backward pass per tile shape, installs the
        fastest and returns it."""
        return _s.srn_autotune(self.handle, _stream_ptr(stream), xyz.data_ptr(), target.data_ptr(), offsets,
                               _s.SRN_DENSITY if density else 0, reps)

    def step(self, density: bool = False, stream=None) -> None:
        _s.srn_step(self.handle, _stream_ptr(stream), _s.SRN_DENSITY if density else 0)

    def sample_points(self, seed: int, step: int, offsets, xyz: torch.Tensor | None = None, stream=None):
        if xyz is None:
            xyz = torch.empty((offsets[-1], 3), dtype=torch.float32, device=self.device)
        _s.srn_sample_points(self.handle, _stream_ptr(stream), seed, step, None, offsets, xyz.data_ptr())
        return xyz

    def sample_target(self, volume, boxes, xyz, offsets, target=None, stream=None):
        """v(x) of every point; `volume` is a float32 [z][y][x] tensor or a TiledVolume."""
        if target is None:
            target = torch.empty(xyz.shape[0], dtype=torch.float32, device=self.device)
        if isinstance(volume, TiledVolume):
            _s.srn_sample_target_tiled(self.handle, _stream_ptr(stream), volume.data.data_ptr(), volume.dims,
                                       np.asarray(boxes).ravel(), xyz.data_ptr(), offsets, target.data_ptr())
            return target
        dims = [volume.shape[2], volume.shape[1], volume.shape[0]]
        _s.srn_sample_target(self.handle, _stream_ptr(stream), volume.data_ptr(), dims,
                             np.asarray(boxes).ravel(), xyz.data_ptr(), offsets, target.data_ptr())
        return target

    def set_schedule(self, delay_iters=500, density_window=1000, density_rel=1e-4, density_frac=0.8,
                     total_iters=50000, plateau_window=500, plateau_rel=1e-4, plateau_factor=0.1,
                     plateau_max=3) -> None:
        """The paper's training routine (Sec. 4.3.2 and 5.2), applied on the device by
        train_step(..., schedule=True); defaults are the paper's values."""
        _s.srn_set_schedule(self.handle, _s.Schedule(delay_iters, density_window, density_rel, density_frac,
                                                     total_iters, plateau_window, plateau_rel, plateau_factor,
                                                     plateau_max))

    def read_schedule(self, stream=None) -> list:
        return _s.srn_read_schedule(self.handle, _stream_ptr(stream), self.n_bricks)

    def rebalanced_offsets(self, base_counts, min_points: int = 1024, stream=None) -> list:
        """Batch offsets that give the finished bricks' shares to the bricks still
        training (srn_rebalance on the device routine's state; synchronises `stream`)."""
        return _s.srn_rebalance(base_counts, self.read_schedule(stream), min_points)

    def train_step(self, seed, volume, boxes, offsets, density, xyz, target, stream=None, schedule=False):
        """One srn_train_step; `volume` is a float32 [z][y][x] tensor or a TiledVolume."""
        flags = _s.SRN_SCHEDULE if schedule else (_s.SRN_DENSITY if density else 0)
        if isinstance(volume, TiledVolume):
            dims, ptr = volume.dims, volume.data.data_ptr()
            flags |= _s.SRN_VOLUME_TILED
        else:
            dims, ptr = [volume.shape[2], volume.shape[1], volume.shape[0]], volume.data_ptr()
        _s.srn_train_step(self.handle, _stream_ptr(stream), seed, ptr, dims,
                          np.asarray(boxes).ravel(), offsets, flags,
                          xyz.data_ptr(), target.data_ptr(), self.losses.data_ptr())
        return self.losses

    def render(self, cam: dict, lut: torch.Tensor, vmin, vmax, width, height, samples, grid, boxes,
               vox, rgba=None, stream=None):
        if rgba is None:
            rgba = torch.empty((height, width, 4), dtype=torch.float32, device=self.device)
        c = _s.Camera((ct_f3(cam["eye"])), ct_f3(cam["forward"]), ct_f3(cam["right"]), ct_f3(cam["up"]),
                      float(cam["scale"]), 1 if cam["ortho"] else 0)
        _s.srn_render(self.handle, _stream_ptr(stream), c, lut.data_ptr(), vmin, vmax, width, height,
                      samples, grid, np.asarray(boxes).ravel(), vox, rgba.data_ptr())
        return rgba

    def render_progressive(self, cam: dict, lut: torch.Tensor, vmin, vmax, width, height, samples, grid, boxes,
                           vox, first, count, rgba, preview=None, stream=None):
        """One pass of progressive rendering (srn_render_progressive): pixels first ..
        first + count - 1 of the image-hierarchy order into rgba, and, if preview is
        given, the in-progress image after them."""
        c = _s.Camera((ct_f3(cam["eye"])), ct_f3(cam["forward"]), ct_f3(cam["right"]), ct_f3(cam["up"]),
                      float(cam["scale"]), 1 if cam["ortho"] else 0)
        _s.srn_render_progressive(self.handle, _stream_ptr(stream), c, lut.data_ptr(), vmin, vmax, width, height,
                                  samples, grid, np.asarray(boxes).ravel(), vox, first, count, rgba.data_ptr(),
                                  preview.data_ptr() if preview is not None else None)
        return rgba

    # ------------------------------------------------------------------ checkpoints
    def save(self, path, stream=None) -> None:
        """Write a checkpoint: parameters, Adam moments, data ranges and the library's
        training state (sampler step, Adam counts), enough to resume bit for bit."""
        torch.cuda.current_stream().synchronize()
        s = self.shape
        np.savez(path, params=self.params.cpu().numpy(), adam_m=self.adam_m.cpu().numpy(),
                 adam_v=self.adam_v.cpu().numpy(), range=self.range.cpu().numpy(),
                 state=np.frombuffer(_s.srn_save_state(self.handle, _stream_ptr(stream)), dtype=np.uint8),
                 shape=np.array([s.n_grids, s.res, s.channels, s.hidden, self.n_bricks, int(self.bf16)]))

    def load(self, path, stream=None) -> None:
        """Resume from a checkpoint written by save() for the same shape and precision."""
        z = np.load(path)
        s = self.shape
        want = np.array([s.n_grids, s.res, s.channels, s.hidden, self.n_bricks, int(self.bf16)])
        if not np.array_equal(z["shape"], want):
            raise ValueError(f"checkpoint of shape {z['shape'].tolist()}, model is {want.tolist()}")
        for name, t in (("params", self.params), ("adam_m", self.adam_m), ("adam_v", self.adam_v), ("range", self.range)):
            t.copy_(torch.as_tensor(z[name]))
        _s.srn_load_state(self.handle, _stream_ptr(stream), z["state"].tobytes())
        _s.srn_sync_shadow(self.handle, _stream_ptr(stream))

    def decode(self, grid, boxes, vox, out=None, stream=None):
        """f at every voxel of a vox^3 volume through the brick decomposition (srn_decode)."""
        if out is None:
            out = torch.empty((vox, vox, vox), dtype=torch.float32, device=self.device)
        _s.srn_decode(self.handle, _stream_ptr(stream), grid, np.asarray(boxes).ravel(), vox, out.data_ptr())
        return out

    def status(self, stream=None) -> None:
        _s.srn_get_status(self.handle, _stream_ptr(stream))


def ct_f3(v):
    import ctypes as ct
    return (ct.c_float * 3)(*[float(a) for a in v])


class APMGSRNFunction(torch.autograd.Function):
    """f = APMGSRN(x) with the flat parameter tensor as the differentiable input.

    ``params`` is a float32 tensor in the model's flat layout (``model.params``
    itself, a clone of it, or ``model.pack(...)``).  The library evaluates the
    model held by its handle, so forward first makes the model hold ``params``:
    unless ``params`` is ``model.params`` itself, its values are copied into
    ``model.params`` and the BF16 shadow is re-derived.  The model keeps those
    values afterwards, and backward differentiates at them.

    forward runs ``srn_forward``; backward runs ``srn_backward`` with
    ``SRN_UPSTREAM`` (the incoming dL/df per point) and returns the flat
    gradient for the parameters (no gradient for the coordinates).  With
    grad_transforms the G part is the full gradient of f through Eq. 1-2
    (SRN_REC_DG); without it G's part is zero, as in the paper's training, where
    only L_den moves G."""

    @staticmethod
    def forward(ctx, xyz, params, model: SRN, offsets, grad_transforms: bool = False):
        if params.shape != model.params.shape or params.dtype != torch.float32 or params.device != model.params.device:
            raise ValueError(f"params must be a float32 tensor of shape {tuple(model.params.shape)} on "
                             f"{model.params.device} (the model's flat layout)")
        if params.data_ptr() != model.params.data_ptr():
            model.params.copy_(params.detach())
            model.sync_shadow()
        ctx.model, ctx.offsets, ctx.rec_dg = model, offsets, grad_transforms
        ctx.save_for_backward(xyz)
        return model.forward(xyz, offsets)

    @staticmethod
    def backward(ctx, grad_f):
        (xyz,) = ctx.saved_tensors
        g = grad_f.contiguous().to(torch.float32)
        ctx.model.backward(xyz, g, ctx.offsets, upstream=True, rec_dg=ctx.rec_dg)
        return None, ctx.model.grads.clone(), None, None, None
