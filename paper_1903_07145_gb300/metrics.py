"""Parameter error of a recovered scene against its ground truth.

Relative L2 error over the normalised parameters that the images determine:
diffuse albedo, specular albedo and emission of every segment seen by at
least one pixel centre, plus roughness where the true specular albedo has a
luminance of at least 0.05 (elsewhere the images barely depend on it).
Visibility comes from the library's ray casting of pixel-centre camera rays.
"""
from __future__ import annotations

import numpy as np
import torch

LUM = np.array([0.2126, 0.7152, 0.0722])


def pixel_center_rays(cam):
    """Origins and unit directions of the camera's pixel-centre rays."""
    W, H = cam.width, cam.height
    th = np.tan(0.5 * np.radians(cam.fov_y_deg))
    px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    dc = np.stack([(2 * px / W - 1) * th * W / H, (1 - 2 * py / H) * th, -np.ones_like(px)], -1).reshape(-1, 3)
    M = np.asarray(cam.cam_to_world, np.float64)
    d = dc @ M[:, :3].T
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(M[:, 3], d.shape)
    return o.astype(np.float32), d.astype(np.float32)


def visible_segments(tracer, scene) -> np.ndarray:
    """Boolean (S,) mask of segments hit by a pixel-centre ray of any view."""
    seen = np.zeros(scene.n_segments, bool)
    for cam in scene.cameras:
        o, d = pixel_center_rays(cam)
        tri = tracer.trace_rays(torch.from_numpy(o), torch.from_numpy(d))[0].cpu().numpy()
        hit = tri[tri >= 0]
        seen[np.unique(scene.tri_segment[hit])] = True
    return seen


def identifiable_mask(gt: np.ndarray, visible: np.ndarray, roughness_min_lum: float = 0.05) -> np.ndarray:
    m = np.zeros_like(gt, bool)
    m[visible, 0:6] = True
    m[visible, 7:10] = True
    m[visible, 6] = (gt[visible, 3:6] @ LUM) >= roughness_min_lum
    return m


def param_error(params: np.ndarray, gt: np.ndarray, mask: np.ndarray) -> float:
    d = (np.asarray(params, np.float64) - np.asarray(gt, np.float64))[mask]
    return float(np.linalg.norm(d) / np.linalg.norm(np.asarray(gt, np.float64)[mask]))


def triangle_pixel_errors(tracer, scene, image, target) -> np.ndarray:
    """Per triangle (original ids): the mean over the pixels whose centre ray
    hits it of the squared RGB residual |I - T|^2 (App. B subdivides the
    triangles where this average is high); NaN where no pixel centre lands."""
    img = np.asarray(image.cpu() if hasattr(image, "cpu") else image, np.float64).reshape(-1, 3)
    tgt = np.asarray(target.cpu() if hasattr(target, "cpu") else target, np.float64).reshape(-1, 3)
    sums = np.zeros(scene.n_tri)
    cnt = np.zeros(scene.n_tri)
    off = 0
    for cam in scene.cameras:
        n = cam.width * cam.height
        o, d = pixel_center_rays(cam)
        tri = tracer.trace_rays(torch.from_numpy(o), torch.from_numpy(d))[0].cpu().numpy()
        r = ((img[off:off + n] - tgt[off:off + n]) ** 2).sum(axis=1)
        hit = tri >= 0
        np.add.at(sums, tri[hit], r[hit])
        np.add.at(cnt, tri[hit], 1.0)
        off += n
    with np.errstate(invalid="ignore", divide="ignore"):
        return sums / cnt
