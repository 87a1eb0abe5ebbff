"""Seeded synthetic inputs: textures, scenes (per-pixel UV and UV Jacobian), views.

This module holds none of the filtering method's arithmetic.  It only makes
inputs, the same arrays for the CUDA path and for the CPU oracle:

* block-compressed textures with uniformly random endpoints and indices,
* a procedural RGBA target (gradient noise + checker edges) and a simple block
  encoder for it (per-block min/max endpoints, nearest palette index),
* screen-space UV and UV Jacobians from ray/plane intersection (FP64, rounded
  to FP32 at the end): the magnified plane, the perspective ground plane with
  tilted quads, the rotated head-on quad of the paper's threshold study
  (supplemental Sec. 3.1, first scene), and batches of uneven views.

The paper's own scenes (Falcor meshes) and textures (4096^2 photo textures) are
not available; these stand in for them with the sizes and magnification ranges
of the workloads the library is measured on.

Jacobian layout per pixel: (du/dx, dv/dx, du/dy, dv/dy) in normalised UV per
pixel.  Magnification of a pixel = 1 / max column norm of the Jacobian in
texels per pixel.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_TEXTURE = 1
SEED_SCENE = 2
SEED_STF = 0
SEED_TRAIN = 3


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed, stream]))


# ---------------------------------------------------------------------------
# Textures
# ---------------------------------------------------------------------------
def random_blocks(Wt: int, Ht: int, seed: int = SEED_TEXTURE) -> np.ndarray:
    """(Ht/4)*(Wt/4) blocks of 8 bytes: u16 c0, u16 c1, u32 index bits, all
    uniform random.  Returned as a flat uint8 array (little endian)."""
    assert Wt % 4 == 0 and Ht % 4 == 0
    nb = (Wt // 4) * (Ht // 4)
    g = _rng(seed, 17)
    c0 = g.integers(0, 1 << 16, nb, dtype=np.uint32).astype("<u2")
    c1 = g.integers(0, 1 << 16, nb, dtype=np.uint32).astype("<u2")
    ix = g.integers(0, 1 << 32, nb, dtype=np.uint64).astype("<u4")
    rec = np.zeros(nb, dtype=[("c0", "<u2"), ("c1", "<u2"), ("ix", "<u4")])
    rec["c0"], rec["c1"], rec["ix"] = c0, c1, ix
    return rec.view(np.uint8).copy()


def _fade(t):
    return t * t * t * (t * (t * 6 - 15) + 10)


def gradient_noise(n: int, freq: int, g: np.random.Generator) -> np.ndarray:
    """n x n tileable 2-D gradient noise with a freq x freq lattice, in about [-0.7, 0.7]."""
    ang = g.uniform(0, 2 * np.pi, (freq, freq))
    gx, gy = np.cos(ang).astype(np.float32), np.sin(ang).astype(np.float32)
    coords = (np.arange(n, dtype=np.float32) + 0.5) * (freq / n)
    i0 = np.floor(coords).astype(np.int64)
    f = coords - i0
    i1 = (i0 + 1) % freq
    i0 = i0 % freq
    fx, fy = f[None, :], f[:, None]
    ux, uy = _fade(fx), _fade(fy)

    def corner(iy, ix, ox, oy):
        return gx[iy[:, None], ix[None, :]] * (fx - ox) + gy[iy[:, None], ix[None, :]] * (fy - oy)

    n00 = corner(i0, i0, 0.0, 0.0)
    n10 = corner(i0, i1, 1.0, 0.0)
    n01 = corner(i1, i0, 0.0, 1.0)
    n11 = corner(i1, i1, 1.0, 1.0)
    nx0 = n00 + ux * (n10 - n00)
    nx1 = n01 + ux * (n11 - n01)
    return (nx0 + uy * (nx1 - nx0)).astype(np.float32)


def _gradient_noise_torch(n: int, freq: int, g: np.random.Generator, device):
    """gradient_noise evaluated with torch on `device` (same lattice draws)."""
    import torch
    ang = g.uniform(0, 2 * np.pi, (freq, freq))
    gx = torch.from_numpy(np.cos(ang).astype(np.float32)).to(device)
    gy = torch.from_numpy(np.sin(ang).astype(np.float32)).to(device)
    coords = (torch.arange(n, dtype=torch.float32, device=device) + 0.5) * (freq / n)
    i0 = torch.floor(coords).long()
    f = coords - i0
    i1 = (i0 + 1) % freq
    i0 = i0 % freq
    fx, fy = f[None, :], f[:, None]
    ux, uy = _fade(fx), _fade(fy)

    def corner(iy, ix, ox, oy):
        return gx[iy[:, None], ix[None, :]] * (fx - ox) + gy[iy[:, None], ix[None, :]] * (fy - oy)

    n00 = corner(i0, i0, 0.0, 0.0)
    n10 = corner(i0, i1, 1.0, 0.0)
    n01 = corner(i1, i0, 0.0, 1.0)
    n11 = corner(i1, i1, 1.0, 1.0)
    nx0 = n00 + ux * (n10 - n00)
    nx1 = n01 + ux * (n11 - n01)
    return nx0 + uy * (nx1 - nx0)


def procedural_rgba8(n: int, seed: int = SEED_TEXTURE, octaves: int = 6, base_freq: int = 8,
                     device=None) -> np.ndarray:
    """n x n RGBA8 target: per channel 6 octaves of gradient noise plus a
    checker pattern with sharp edges; alpha 255.  With `device` (a torch
    device) the noise is evaluated there; the lattice draws are the same."""
    g = _rng(seed, 29)
    checker_cells = 16
    if device is not None:
        import torch
        yy, xx = torch.meshgrid(torch.arange(n, device=device), torch.arange(n, device=device), indexing="ij")
        checker = (((xx * checker_cells) // n + (yy * checker_cells) // n) % 2).float()
        out = torch.zeros((n, n, 4), dtype=torch.uint8, device=device)
        for ch in range(3):
            acc = torch.zeros((n, n), dtype=torch.float32, device=device)
            amp, freq = 0.5, base_freq
            for _ in range(octaves):
                acc += amp * _gradient_noise_torch(n, min(freq, n), g, device)
                amp *= 0.5
                freq *= 2
            tint = g.uniform(0.15, 0.35)
            img = (0.5 + 0.8 * acc + tint * (checker - 0.5)).clamp(0.0, 1.0)
            out[..., ch] = torch.round(img * 255.0).to(torch.uint8)
        out[..., 3] = 255
        return out.cpu().numpy()
    img = np.zeros((n, n, 4), np.float32)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    checker = (((xx * checker_cells) // n + (yy * checker_cells) // n) % 2).astype(np.float32)
    for ch in range(3):
        acc = np.zeros((n, n), np.float32)
        amp, freq = 0.5, base_freq
        for _ in range(octaves):
            acc += amp * gradient_noise(n, min(freq, n), g)
            amp *= 0.5
            freq *= 2
        tint = g.uniform(0.15, 0.35)
        img[..., ch] = 0.5 + 0.8 * acc + tint * (checker - 0.5)
    img = np.clip(img, 0.0, 1.0)
    out = np.rint(img * 255.0).astype(np.uint8)
    out[..., 3] = 255
    return out


def encode_blocks(rgba8: np.ndarray) -> np.ndarray:
    """Simple encoder into the 8-byte block format: per 4x4 block the endpoints
    are the per-channel min (c0) and max (c1) quantised to RGB565; each texel
    takes the palette entry nearest in squared RGB distance.  The palette is
    built here with the format's published rules (bit replication, 1/3 and 2/3
    points rounded) only to choose indices; decoding is not done here."""
    Ht, Wt = rgba8.shape[:2]
    assert Wt % 4 == 0 and Ht % 4 == 0
    blk = rgba8[..., :3].astype(np.int32).reshape(Ht // 4, 4, Wt // 4, 4, 3).transpose(0, 2, 1, 3, 4)
    blk = blk.reshape(Ht // 4, Wt // 4, 16, 3)
    lo, hi = blk.min(axis=2), blk.max(axis=2)

    def to565(c):
        r = np.clip((c[..., 0] * 31 + 127) // 255, 0, 31)
        gg = np.clip((c[..., 1] * 63 + 127) // 255, 0, 63)
        b = np.clip((c[..., 2] * 31 + 127) // 255, 0, 31)
        return (r << 11) | (gg << 5) | b

    def expand(c):
        r5, g6, b5 = (c >> 11) & 31, (c >> 5) & 63, c & 31
        return np.stack([(r5 << 3) | (r5 >> 2), (g6 << 2) | (g6 >> 4), (b5 << 3) | (b5 >> 2)], axis=-1)

    c0, c1 = to565(lo), to565(hi)
    e0, e1 = expand(c0), expand(c1)
    pal = np.stack([e0, e1, (2 * e0 + e1 + 1) // 3, (e0 + 2 * e1 + 1) // 3], axis=2)  # [by,bx,4,3]
    d = ((blk[:, :, :, None, :] - pal[:, :, None, :, :]) ** 2).sum(-1)  # [by,bx,16,4]
    sel = d.argmin(-1).astype(np.uint64)  # [by,bx,16]
    bits = np.zeros(sel.shape[:2], np.uint64)
    for k in range(16):
        bits |= sel[:, :, k] << np.uint64(2 * k)
    nb = (Ht // 4) * (Wt // 4)
    rec = np.zeros(nb, dtype=[("c0", "<u2"), ("c1", "<u2"), ("ix", "<u4")])
    rec["c0"] = c0.reshape(-1).astype(np.uint16)
    rec["c1"] = c1.reshape(-1).astype(np.uint16)
    rec["ix"] = bits.reshape(-1).astype(np.uint32)
    return rec.view(np.uint8).copy()


# ---------------------------------------------------------------------------
# Scenes
# ---------------------------------------------------------------------------
@dataclass
class Scene:
    """One view: per-pixel uv [H,W,2] f32, jac [H,W,4] f32, coverage [H,W] u8 or None."""
    W: int
    H: int
    uv: np.ndarray
    jac: np.ndarray
    coverage: np.ndarray | None
    name: str = ""
    meta: dict = field(default_factory=dict)

    def magnification(self, Wt: int, Ht: int) -> np.ndarray:
        j = self.jac.astype(np.float64)
        rx = np.hypot(j[..., 0] * Wt, j[..., 1] * Ht)
        ry = np.hypot(j[..., 2] * Wt, j[..., 3] * Ht)
        with np.errstate(divide="ignore"):
            return 1.0 / np.maximum(rx, ry)


def magnified_plane(W: int = 128, H: int = 128, Wt: int = 64, Ht: int = 64, scale: float = 0.25,
                    seed: int = SEED_SCENE) -> Scene:
    """Screen-aligned plane: texel position = pixel * scale + jitter, jitter
    uniform in [0, scale) texels per pixel and axis (uniform 1/scale
    magnification)."""
    g = _rng(seed, 1)
    py, px = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    jx = g.uniform(0.0, scale, (H, W))
    jy = g.uniform(0.0, scale, (H, W))
    uv = np.stack([(px * scale + jx) / Wt, (py * scale + jy) / Ht], axis=-1).astype(np.float32)
    jac = np.zeros((H, W, 4), np.float32)
    jac[..., 0] = scale / Wt
    jac[..., 3] = scale / Ht
    return Scene(W, H, uv, jac, None, name=f"plane{W}x{H}_m{1/scale:g}")


def _camera_rays(W, H, fov_y_deg, pitch_deg, yaw_deg=0.0):
    """World-space ray directions for pixel centres and their derivatives per pixel."""
    f = (H / 2) / math.tan(math.radians(fov_y_deg) / 2)
    py, px = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    dc = np.stack([px + 0.5 - W / 2, -(py + 0.5 - H / 2), np.full_like(px, f)], axis=-1)
    p, yw = math.radians(pitch_deg), math.radians(yaw_deg)
    # pitch about x (negative looks down), then yaw about y
    Rx = np.array([[1, 0, 0], [0, math.cos(p), -math.sin(p)], [0, math.sin(p), math.cos(p)]])
    Ry = np.array([[math.cos(yw), 0, math.sin(yw)], [0, 1, 0], [-math.sin(yw), 0, math.cos(yw)]])
    R = Ry @ Rx
    d = dc @ R.T
    ddx = R @ np.array([1.0, 0.0, 0.0])
    ddy = R @ np.array([0.0, -1.0, 0.0])
    return d, ddx, ddy


def _hit_plane(C, d, ddx, ddy, O, U, V, ku, kv, u0, v0, LU, LV):
    """Intersect rays with the rectangle O + a U + b V, a in [0,LU], b in [0,LV].
    Texture coordinate (u, v) = (u0 + ku a, v0 + kv b).  Returns t, uv, jac, valid."""
    N = np.cross(U, V)
    dn = d @ N
    k = float((O - C) @ N)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = k / dn
        X = C + t[..., None] * d
        a = (X - O) @ U
        b = (X - O) @ V
        valid = (t > 1e-6) & (a >= 0) & (a <= LU) & (b >= 0) & (b <= LV) & np.isfinite(t)
        dXdx = k * (ddx[None, None, :] * dn[..., None] - d * (ddx @ N)) / (dn ** 2)[..., None]
        dXdy = k * (ddy[None, None, :] * dn[..., None] - d * (ddy @ N)) / (dn ** 2)[..., None]
    uv = np.stack([u0 + ku * a, v0 + kv * b], axis=-1)
    jac = np.stack([ku * (dXdx @ U), kv * (dXdx @ V), ku * (dXdy @ U), kv * (dXdy @ V)], axis=-1)
    return t, uv, jac, valid


def ground_plane_with_quads(W: int = 1920, H: int = 1080, Wt: int = 2048, Ht: int = 2048,
                            seed: int = SEED_SCENE, n_quads: int = 3, pitch_deg: float = 33.0,
                            fov_y_deg: float = 50.0, cam_height: float = 1.0, extent: float = 40.0) -> Scene:
    """Perspective ground plane (magnification from about 32 near the camera
    down into minification towards the horizon) plus n seeded tilted, rotated
    quads whose texture scale is drawn log-uniform so that their
    magnification spans [0.5, 32].  Sky pixels have coverage 0."""
    g = _rng(seed, 2)
    C = np.array([0.0, cam_height, 0.0])
    d, ddx, ddy = _camera_rays(W, H, fov_y_deg=fov_y_deg, pitch_deg=pitch_deg)
    best_t = np.full((H, W), np.inf)
    uv = np.zeros((H, W, 2))
    jac = np.zeros((H, W, 4))
    cov = np.zeros((H, W), np.uint8)
    # ground plane y = 0: O at (-L/2, 0, 0), axes x and z; one texture copy over L x L
    L = extent
    O = np.array([-L / 2, 0.0, 0.3])
    U, V = np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])
    # rectangle U x V has normal U x V = (0,-1,0); intersection formula is orientation-free
    t, uvp, jp, ok = _hit_plane(C, d, ddx, ddy, O, U, V, 1.0 / L, 1.0 / L, 0.0, 0.0, L, L)
    sel = ok & (t < best_t)
    best_t[sel], uv[sel], jac[sel], cov[sel] = t[sel], uvp[sel], jp[sel], 1
    for q in range(n_quads):
        # a quad centred on a random screen point, between the camera and the ground
        spx, spy = g.uniform(0.15 * W, 0.85 * W), g.uniform(0.15 * H, 0.75 * H)
        dq = d[int(spy), int(spx)]
        dq = dq / np.linalg.norm(dq)
        t_ground = cam_height / -dq[1] if dq[1] < 0 else 10.0
        dist = g.uniform(0.35, 0.7) * min(t_ground, 10.0)
        center = C + dist * dq
        size = 0.45 * dist
        yaw, tilt, roll = g.uniform(-0.8, 0.8), g.uniform(-0.6, 0.6), g.uniform(0, 2 * np.pi)
        Rz = np.array([[math.cos(roll), -math.sin(roll), 0], [math.sin(roll), math.cos(roll), 0], [0, 0, 1]])
        Rx = np.array([[1, 0, 0], [0, math.cos(tilt), -math.sin(tilt)], [0, math.sin(tilt), math.cos(tilt)]])
        Ry = np.array([[math.cos(yaw), 0, math.sin(yaw)], [0, 1, 0], [-math.sin(yaw), 0, math.cos(yaw)]])
        R = Ry @ Rx @ Rz
        Uq, Vq = R @ np.array([1.0, 0, 0]), R @ np.array([0, 1.0, 0])
        Oq = center - 0.5 * size * Uq - 0.5 * size * Vq
        # texture scale: texels per world unit drawn log-uniform, clipped to one texture copy
        m_target = math.exp(g.uniform(math.log(1.0), math.log(32.0)))
        # pixel footprint at that distance ~ dist / f (f in pixels)
        f = (H / 2) / math.tan(math.radians(fov_y_deg) / 2)
        texels_per_unit = f / (dist * m_target)
        k = texels_per_unit / Wt
        k = min(k, 1.0 / size)
        u0 = g.uniform(0.0, max(1e-6, 1.0 - k * size))
        v0 = g.uniform(0.0, max(1e-6, 1.0 - k * size))
        t, uvq, jq, ok = _hit_plane(C, d, ddx, ddy, Oq, Uq, Vq, k, k, u0, v0, size, size)
        sel = ok & (t < best_t)
        best_t[sel], uv[sel], jac[sel], cov[sel] = t[sel], uvq[sel], jq[sel], 1
    uv[cov == 0] = 0.0
    jac[cov == 0] = 0.0
    return Scene(W, H, uv.astype(np.float32), jac.astype(np.float32), cov,
                 name=f"ground+{n_quads}quads_{W}x{H}", meta={"texture": (Wt, Ht)})


def rotated_quad_tiles(m: float, degrees, n_phase: int, tile_w: int = 8, tile_h: int = 4,
                       Wt: int = 4096, Ht: int = 4096, seed: int = SEED_SCENE) -> Scene:
    """The threshold study of the paper (Fig. 4): a head-on quad rotated by
    r degrees about the view axis and magnified m times.  One warp tile per
    (rotation, sub-texel phase): pixel centre p (in pixels, relative to the
    tile) maps to texel position R(r) p / m + o, o a random offset.  Tiles are
    stacked vertically (frame width = tile_w)."""
    g = _rng(seed, 3)
    degrees = np.atleast_1d(np.asarray(degrees, np.float64))
    ntiles = degrees.size * n_phase
    H = ntiles * tile_h
    W = tile_w
    ly, lx = np.meshgrid(np.arange(tile_h, dtype=np.float64) + 0.5, np.arange(tile_w, dtype=np.float64) + 0.5,
                         indexing="ij")
    uv = np.zeros((H, W, 2))
    jac = np.zeros((H, W, 4))
    tile = 0
    for r in degrees:
        c, s = math.cos(math.radians(r)), math.sin(math.radians(r))
        for _ in range(n_phase):
            o = g.uniform(1024.0, 1025.0, 2)
            X = (c * lx - s * ly) / m + o[0]
            Y = (s * lx + c * ly) / m + o[1]
            rows = slice(tile * tile_h, (tile + 1) * tile_h)
            uv[rows, :, 0] = X / Wt
            uv[rows, :, 1] = Y / Ht
            jac[rows, :, 0] = c / m / Wt
            jac[rows, :, 1] = s / m / Ht
            jac[rows, :, 2] = -s / m / Wt
            jac[rows, :, 3] = c / m / Ht
            tile += 1
    return Scene(W, H, uv.astype(np.float32), jac.astype(np.float32), None, name=f"rotquad_m{m:g}")


def perspective_view(W: int, H: int, Wt: int, Ht: int, m_lo: float, m_hi: float, seed: int,
                     view: int = 0) -> Scene:
    """A view of one textured plane whose magnification runs roughly
    log-uniformly from m_hi (near the bottom of the frame) to m_lo (top): the
    plane is tilted so the pixel footprint grows geometrically with the row."""
    g = _rng(seed, 100 + view)
    rot = g.uniform(0, 2 * np.pi)
    u0, v0 = g.uniform(0.2, 0.8, 2)
    py, px = np.meshgrid(np.arange(H, dtype=np.float64) + 0.5, np.arange(W, dtype=np.float64) + 0.5,
                         indexing="ij")
    # texels per pixel rho(y) = exp(a + b*y) from 1/m_hi (bottom) to 1/m_lo (top)
    a_bot, a_top = math.log(1.0 / m_hi), math.log(1.0 / m_lo)
    yn = 1.0 - py / H                    # 0 at bottom, 1 at top
    lrho = a_bot + (a_top - a_bot) * yn  # log texels-per-pixel
    rho = np.exp(lrho)
    # texel-space position: integrate rho along y, scale x by rho too (isotropic)
    k = (a_top - a_bot) / H
    # d/dy of Y must be -rho (moving up increases distance): Y = -(rho - rho_bot)/(-k) ...
    with np.errstate(divide="ignore", invalid="ignore"):
        Yt = (np.exp(a_bot) - rho) / k if abs(k) > 1e-12 else -rho * py
    Xt = (px - W / 2) * rho
    c, s = math.cos(rot), math.sin(rot)
    X = c * Xt - s * Yt
    Y = s * Xt + c * Yt
    dXt_dx, dXt_dy = rho, (px - W / 2) * rho * (-k)
    dYt_dx, dYt_dy = np.zeros_like(rho), rho
    # d/dy of rho = rho * (-k) since yn decreases with py
    jxx = c * dXt_dx - s * dYt_dx
    jyx = s * dXt_dx + c * dYt_dx
    jxy = c * dXt_dy - s * dYt_dy
    jyy = s * dXt_dy + c * dYt_dy
    uv = np.stack([u0 + X / Wt, v0 + Y / Ht], axis=-1)
    jac = np.stack([jxx / Wt, jyx / Ht, jxy / Wt, jyy / Ht], axis=-1)
    cov = ((uv[..., 0] >= 0) & (uv[..., 0] <= 1) & (uv[..., 1] >= 0) & (uv[..., 1] <= 1)).astype(np.uint8)
    uv[cov == 0] = 0.0
    jac[cov == 0] = 0.0
    return Scene(W, H, uv.astype(np.float32), jac.astype(np.float32), cov, name=f"view{view}_{W}x{H}")


def uneven_views(n_views: int = 64, seed: int = SEED_SCENE, max_w: int = 3840, max_h: int = 2160,
                 min_w: int = 256, min_h: int = 256, m_lo: float = 0.25, m_hi: float = 64.0,
                 textures=((2048, 2048), (4096, 4096))):
    """Sizes uniform in [min, max] per axis, each view a tilted plane with its
    own magnification range inside [m_lo, m_hi] (log-uniform endpoints) and
    texture alternating between the given texture sizes.  Returns a list of
    (Scene, texture_index)."""
    g = _rng(seed, 5)
    views = []
    for v in range(n_views):
        W = int(g.integers(min_w, max_w + 1))
        H = int(g.integers(min_h, max_h + 1))
        lo, hi = sorted(np.exp(g.uniform(math.log(m_lo), math.log(m_hi), 2)))
        ti = v % len(textures)
        Wt, Ht = textures[ti]
        views.append((perspective_view(W, H, Wt, Ht, float(lo), float(hi), seed, view=v), ti))
    return views
