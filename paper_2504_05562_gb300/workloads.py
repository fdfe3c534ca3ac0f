"""Seeded synthetic inputs: materials, views and view batches.

This module produces the bytes and camera matrices that BOTH the GPU library and the CPU
oracle consume. It holds none of the filtering method's arithmetic: noise and brick
patterns make texels, a pinhole camera makes a screen->texture homography, and encoders
turn FP32 texels into the stored formats. Everything is deterministic given the seed.

The paper's scenes use photographed texture sets that are not available here; these stand
in for them with the mix its error analysis cares about (Section 3): smooth low-frequency
regions (value noise, fBm) plus sharp high-contrast edges (a brick-and-mortar mask).

Formats: FP32=0, FP16=1, BF16=2, E4M3=3, UNORM8=4 (the codes of the C interface).
"""
from __future__ import annotations

import functools
import math

import numpy as np

FP32, FP16, BF16, E4M3, UNORM8 = 0, 1, 2, 3, 4
BILINEAR, BSPLINE3 = 0, 1
LIGHT_DIR = tuple((np.array([0.3, 1.0, 0.2]) / np.linalg.norm([0.3, 1.0, 0.2])).tolist())

# --------------------------------------------------------------------------- noise


def _hash2(ix, iy, seed):
    """32-bit integer hash of lattice points (xorshift-multiply mixing)."""
    h = (ix.astype(np.uint64) * np.uint64(0x8DA6B343) + iy.astype(np.uint64) * np.uint64(0xD8163841)
         + np.uint64(seed) * np.uint64(0xCB1AB31F) + np.uint64(0x165667B1)) & np.uint64(0xFFFFFFFF)
    h = h.astype(np.uint32)
    h ^= h >> np.uint32(16)
    h = (h * np.uint32(0x7FEB352D)) & np.uint32(0xFFFFFFFF)
    h ^= h >> np.uint32(15)
    h = (h * np.uint32(0x846CA68B)) & np.uint32(0xFFFFFFFF)
    h ^= h >> np.uint32(16)
    return h


def value_noise(size, period, seed):
    """Periodic value noise on a size x size grid with lattice spacing `period` texels,
    smoothstep interpolation, values in [0, 1)."""
    n = max(1, size // period)
    lat = _hash2(*np.meshgrid(np.arange(n), np.arange(n), indexing="xy"), seed).astype(np.float64) / 2.0**32
    t = (np.arange(size) + 0.5) / period - 0.5
    i0 = np.floor(t).astype(np.int64)
    f = t - i0
    f = f * f * (3.0 - 2.0 * f)
    a0, a1 = i0 % n, (i0 + 1) % n
    # rows = y, cols = x
    v00 = lat[np.ix_(a0, a0)]
    v01 = lat[np.ix_(a0, a1)]
    v10 = lat[np.ix_(a1, a0)]
    v11 = lat[np.ix_(a1, a1)]
    fy = f[:, None]
    fx = f[None, :]
    return (v00 * (1 - fx) + v01 * fx) * (1 - fy) + (v10 * (1 - fx) + v11 * fx) * fy


def fbm(size, base_period, octaves, seed):
    acc = np.zeros((size, size))
    amp, tot = 0.5, 0.0
    p = base_period
    for o in range(octaves):
        acc += amp * value_noise(size, max(1, p), seed * 131 + o)
        tot += amp
        amp *= 0.5
        p //= 2
    return acc / tot


def _normalise(a):
    lo, hi = a.min(), a.max()
    return (a - lo) / (hi - lo) if hi > lo else np.zeros_like(a)


# --------------------------------------------------------------------------- materials


@functools.lru_cache(maxsize=8)
def noise_rgba(size=64, seed=0):
    """Plain RGBA FP32 texture: 4-octave value noise (lattice periods size/4 ... size/32 for
    size 64: 16, 8, 4, 2; amplitudes 1/2 ... 1/16), each channel normalised to [0, 1]."""
    out = np.zeros((size, size, 4), np.float32)
    for c in range(4):
        acc = np.zeros((size, size))
        for o in range(4):
            acc += 0.5 ** (o + 1) * value_noise(size, max(1, (size // 4) >> o), seed * 977 + c * 31 + o)
        out[..., c] = _normalise(acc)
    return out


def _bricks(size, brick_w, brick_h, mortar):
    y, x = np.mgrid[0:size, 0:size]
    row = y // brick_h
    xs = x + (row % 2) * (brick_w // 2)
    in_mortar = ((xs % brick_w) < mortar) | ((y % brick_h) < mortar)
    brick_id = (row * 7919 + xs // brick_w) % 97
    return in_mortar, brick_id


@functools.lru_cache(maxsize=4)
def brick_material(size=1024, seed=0):
    """Channels (float64, [size, size]): albedo RGB, normal XY, roughness, AO, height.

    Height: 6-octave fBm, with bricks raised above a mortar grid (sharp edges). Albedo: a
    colour ramp over height (mortar grey, bricks red-brown with per-brick tint). Normal: central
    differences of height. Roughness in [0.2, 0.8] and AO in [0.5, 1] follow height and mortar."""
    scale = size / 1024.0
    h = fbm(size, max(2, int(128 * scale)), 6, seed)
    mort, bid = _bricks(size, int(64 * scale), int(32 * scale), max(2, int(4 * scale)))
    height = np.where(mort, 0.15 * h, 0.45 + 0.55 * h)
    tint = (bid.astype(np.float64) / 97.0 - 0.5) * 0.25
    brick_rgb = np.stack([0.55 + tint + 0.3 * h, 0.25 + 0.5 * tint + 0.2 * h, 0.18 + 0.15 * h], -1)
    mortar_rgb = np.stack([0.55 + 0.2 * h] * 3, -1)
    albedo = np.clip(np.where(mort[..., None], mortar_rgb, brick_rgb), 0.0, 1.0)
    strength = 6.0 * scale
    gx = (np.roll(height, -1, 1) - np.roll(height, 1, 1)) * 0.5 * strength
    gy = (np.roll(height, -1, 0) - np.roll(height, 1, 0)) * 0.5 * strength
    n = np.stack([-gx, -gy, np.ones_like(gx)], -1)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    rough = np.clip(np.where(mort, 0.8 - 0.1 * h, 0.2 + 0.5 * (1 - h)), 0.2, 0.8)
    ao = np.clip(np.where(mort, 0.5 + 0.2 * h, 0.75 + 0.25 * h), 0.5, 1.0)
    return np.concatenate([albedo, n[..., :2], rough[..., None], ao[..., None], height[..., None]], -1)


# --------------------------------------------------------------------------- encoders


def encode_fp16(x):
    return np.ascontiguousarray(np.asarray(x, np.float32).astype(np.float16)).view(np.uint16)


def encode_bf16(x):
    """Round-to-nearest-even to bfloat16 (finite inputs)."""
    u = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    r = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return r.astype(np.uint16)


def encode_e4m3(x):
    """Round-to-nearest-even to OCP E4M3 (FN) with saturation to +-448 (via torch's float8)."""
    import torch
    t = torch.from_numpy(np.clip(np.asarray(x, np.float32), -448.0, 448.0).copy())
    return t.to(torch.float8_e4m3fn).view(torch.uint8).numpy()


def encode_unorm8(x):
    return np.clip(np.rint(np.asarray(x, np.float64) * 255.0), 0, 255).astype(np.uint8)


def tile_scales(x, tile, fmt_max):
    """Per (tile, channel) FP32 scales amax / fmt_max, [tiles_y, tiles_x, C]; 1 where amax = 0."""
    h, w, c = x.shape
    ty, tx = (h + tile - 1) // tile, (w + tile - 1) // tile
    s = np.ones((ty, tx, c), np.float32)
    for j in range(ty):
        for i in range(tx):
            a = np.abs(x[j * tile:(j + 1) * tile, i * tile:(i + 1) * tile]).reshape(-1, c).max(0)
            s[j, i] = np.where(a > 0, (a / fmt_max).astype(np.float32), np.float32(1.0))
    return s


def make_material(channels, fmt, scale_tile=64):
    """Encode an FP32/FP64 [h, w, C] array into one plane of `fmt`.
    E4M3 gets per-(64x64 tile, channel) scales; the other formats are stored unscaled."""
    x = np.asarray(channels, np.float32)
    h, w, c = x.shape
    scales = None
    if fmt == FP32:
        data = np.ascontiguousarray(x)
    elif fmt == FP16:
        data = encode_fp16(x)
    elif fmt == BF16:
        data = encode_bf16(x)
    elif fmt == E4M3:
        scales = tile_scales(x.astype(np.float64), scale_tile, 448.0)
        full = np.repeat(np.repeat(scales, scale_tile, 0), scale_tile, 1)[:h, :w]
        data = encode_e4m3(x.astype(np.float64) / full.astype(np.float64))
    elif fmt == UNORM8:
        data = encode_unorm8(x)
    else:
        raise ValueError(fmt)
    return {"width": w, "height": h, "planes": [(fmt, c, np.ascontiguousarray(data))],
            "scales": scales, "scale_tile": scale_tile if scales is not None else 0}


def material_c1(seed=0):
    """64x64 RGBA FP32 value noise."""
    return make_material(noise_rgba(64, seed), FP32)


def material_c2(size=1024, seed=0):
    """Albedo RGBA8 (UNORM8 x 4) plus tangent-space normal XY in RG16F, two planes."""
    m = brick_material(size, seed)
    rgba = np.concatenate([m[..., 0:3], np.ones_like(m[..., :1])], -1)
    return {"width": size, "height": size,
            "planes": [(UNORM8, 4, encode_unorm8(rgba)), (FP16, 2, encode_fp16(m[..., 3:5]))],
            "scales": None, "scale_tile": 0}


def material_c3(fmt, size=2048, seed=0):
    """8 channels (albedo RGB, normal XY, roughness, AO, height) in one plane of `fmt`."""
    return make_material(brick_material(size, seed), fmt)


def decoded_reference(mat):
    """Material texels decoded to float64 [h, w, C] with plain numpy/torch conversions.
    (Used by tests to pin decoders; not an input of either path.)"""
    import torch
    outs = []
    for fmt, c, arr in mat["planes"]:
        a = np.asarray(arr)
        if fmt == FP32:
            v = a.astype(np.float64)
        elif fmt == FP16:
            v = a.view(np.float16).astype(np.float64)
        elif fmt == BF16:
            v = torch.from_numpy(a.astype(np.int16).copy()).view(torch.bfloat16).double().numpy()
        elif fmt == E4M3:
            v = torch.from_numpy(a.copy()).view(torch.float8_e4m3fn).double().numpy()
        else:
            v = a.astype(np.float64) / 255.0
        outs.append(v.reshape(mat["height"], mat["width"], c))
    out = np.concatenate(outs, -1)
    if mat.get("scales") is not None:
        st = mat["scale_tile"]
        full = np.repeat(np.repeat(mat["scales"], st, 0), st, 1)[:mat["height"], :mat["width"]]
        out = (out.astype(np.float32) * full.astype(np.float32)).astype(np.float64)
    return out


# --------------------------------------------------------------------------- views


def _base_view(width, height, H, filt, tile=(8, 4), frame=0, view_id=0):
    return {"width": int(width), "height": int(height),
            "H": [float(np.float32(h)) for h in np.asarray(H, np.float64).ravel()],
            "cam_pos": (0.0, 1.5, 0.0), "plane_to_world": (1.0, 0.0, 0.0, 0.0, 1.0, 0.0),
            "light_dir": LIGHT_DIR, "shading": 0, "ch_albedo": -1, "ch_normal": -1,
            "ch_rough": -1, "ch_ao": -1, "roughness": 0.3, "filter": int(filt), "tile": tuple(tile),
            "frame": int(frame), "view_id": int(view_id)}


def screen_aligned_view(width, height, tex_w, tex_h, mag, filt, origin=None, tile=(8, 4),
                        frame=0, view_id=0, world_per_texel=1.0 / 512.0, cam_height=1.5):
    """Screen-aligned quad at uniform magnification `mag` (pixels per texel per axis):
    uv = (texel origin + (x + 0.5) / mag) / tex_size. A top-down camera at `cam_height` sits above
    the centre of the visible window; world units per texel `world_per_texel`."""
    if origin is None:
        origin = ((tex_w - width / mag) / 2.0, (tex_h - height / mag) / 2.0)
    ox, oy = origin
    H = np.array([[1.0 / (mag * tex_w), 0.0, ox / tex_w],
                  [0.0, 1.0 / (mag * tex_h), oy / tex_h],
                  [0.0, 0.0, 1.0]])
    v = _base_view(width, height, H, filt, tile, frame, view_id)
    cu = (ox + width / (2.0 * mag)) / tex_w
    cv = (oy + height / (2.0 * mag)) / tex_h
    sx, sz = tex_w * world_per_texel, tex_h * world_per_texel
    v["plane_to_world"] = (sx, 0.0, -cu * sx, 0.0, sz, -cv * sz)
    v["cam_pos"] = (0.0, cam_height, 0.0)
    return v


def _perspective_h(width, height, cam_h, fov_y, pitch, s_u, s_v, u_c, v_c):
    """Homography (x+.5, y+.5, 1) -> (u, v, w) for a pinhole camera at (0, cam_h, 0) pitched down
    by `pitch` looking towards +z; uv = (s_u * X + u_c, s_v * Z + v_c) on the ground y = 0."""
    t = math.tan(fov_y / 2.0)
    asp = width / height
    fwd = np.array([0.0, -math.sin(pitch), math.cos(pitch)])
    up = np.array([0.0, math.cos(pitch), math.sin(pitch)])
    right = np.array([1.0, 0.0, 0.0])
    # ray direction d = fwd + sx right + sy up with sx = (2 px / W - 1) t asp, sy = (1 - 2 py / H) t
    A = np.stack([right * (2.0 * t * asp / width), -up * (2.0 * t / height),
                  fwd - right * t * asp + up * t], 1)  # d = A @ (px, py, 1)
    M = np.array([[s_u * cam_h, -u_c, 0.0],
                  [0.0, -v_c, s_v * cam_h],
                  [0.0, -1.0, 0.0]])
    Hm = M @ A
    return Hm / np.abs(Hm).max()


def magnification_field(H, width, height, tex_w, tex_h, samples=33):
    """Area magnification 1 / sqrt(|det d(texel)/d(pixel)|) sampled on a grid (float64)."""
    H = np.asarray(H, np.float64).reshape(3, 3)
    xs = np.linspace(0.5, width - 0.5, samples)
    ys = np.linspace(0.5, height - 0.5, samples)
    X, Y = np.meshgrid(xs, ys)

    def uv(x, y):
        p = H @ np.stack([x.ravel(), y.ravel(), np.ones(x.size)])
        return p[0] / p[2] * tex_w, p[1] / p[2] * tex_h

    e = 1e-3
    u0, v0 = uv(X, Y)
    u1, v1 = uv(X + e, Y)
    u2, v2 = uv(X, Y + e)
    det = ((u1 - u0) * (v2 - v0) - (u2 - u0) * (v1 - v0)) / (e * e)
    return (1.0 / np.sqrt(np.abs(det))).reshape(X.shape)


@functools.lru_cache(maxsize=4)
def _solve_ground_camera(width, height, tex, cam_h, fov_deg, m_lo, m_hi):
    fov = math.radians(fov_deg)

    def field(pitch, dens):
        s = dens / tex
        H = _perspective_h(width, height, cam_h, fov, pitch, s, s, 0.5, 0.5)
        return magnification_field(H, width, height, tex, tex)

    lo, hi = fov / 2.0 + 1e-3, math.radians(89.0)
    for _ in range(60):  # ratio max/min decreases as the camera looks more steeply down
        mid = 0.5 * (lo + hi)
        f = field(mid, 1.0)
        if f.max() / f.min() > m_hi / m_lo:
            lo = mid
        else:
            hi = mid
    pitch = 0.5 * (lo + hi)
    f = field(pitch, 1.0)
    dens = f.min() / m_lo  # magnification scales as 1 / density
    return pitch, dens


def ground_plane_view(width=1920, height=1080, tex=1024, filt=BSPLINE3, cam_h=1.5, fov_deg=60.0,
                      m_lo=2.0, m_hi=32.0, tile=(8, 4), frame=0, view_id=0):
    """Perspective view of the ground plane: camera `cam_h` up, vertical FOV `fov_deg`, pitch and
    texel density solved so the area magnification spans [m_lo, m_hi] over the screen. The visible
    region is centred in the texture."""
    pitch, dens = _solve_ground_camera(width, height, tex, cam_h, fov_deg, m_lo, m_hi)
    s = dens / tex
    fov = math.radians(fov_deg)
    H0 = _perspective_h(width, height, cam_h, fov, pitch, s, s, 0.5, 0.5)
    # centre the visible region in v: shift v_c so the mid-screen depth range sits at 0.5
    corners = np.array([[0.5, 0.5, 1], [width - 0.5, 0.5, 1], [0.5, height - 0.5, 1],
                        [width - 0.5, height - 0.5, 1]]).T
    q = H0 @ corners
    vv = q[1] / q[2]
    v_c = 0.5 - (vv.min() + vv.max()) / 2.0 + 0.5
    H = _perspective_h(width, height, cam_h, fov, pitch, s, s, 0.5, v_c)
    v = _base_view(width, height, H, filt, tile, frame, view_id)
    v["cam_pos"] = (0.0, cam_h, 0.0)
    v["plane_to_world"] = (1.0 / s, 0.0, -0.5 / s, 0.0, 1.0 / s, -v_c / s)
    v["pitch_deg"] = math.degrees(pitch)
    v["texels_per_unit"] = dens
    return v


def with_shading(view, layout):
    """Attach the shading channel map: 'c2' = albedo RGBA + normal XY (roughness 0.3, no AO);
    'c3' = albedo RGB, normal XY, roughness, AO, height."""
    v = dict(view)
    v["shading"] = 1
    if layout == "c2":
        v.update(ch_albedo=0, ch_normal=4, ch_rough=-1, ch_ao=-1, roughness=0.3)
    elif layout == "c3":
        v.update(ch_albedo=0, ch_normal=3, ch_rough=5, ch_ao=6)
    else:
        raise ValueError(layout)
    return v


# --------------------------------------------------------------------------- configs


def config1_view(filt=BILINEAR, tile=(8, 4), frame=0):
    """256x256 screen over a 64x64 texture at uniform 4x."""
    return screen_aligned_view(256, 256, 64, 64, 4.0, filt, origin=(0.0, 0.0), tile=tile, frame=frame)


def config2_view(frame=0, filt=BSPLINE3, tile=(8, 4), width=1920, height=1080, tex=1024):
    return with_shading(ground_plane_view(width, height, tex, filt, tile=tile, frame=frame), "c2")


def config3_view(filt=BILINEAR, tile=(8, 4), frame=0, width=3840, height=2160, tex=2048, mag=4.0):
    return with_shading(screen_aligned_view(width, height, tex, tex, mag, filt, tile=tile, frame=frame), "c3")


RES_CHOICES = ((256, 256), (1280, 720), (1920, 1080), (3840, 2160))


def config5_views(n=64, tex=2048, seed=0, scale=1.0):
    """`n` top-down views: resolution uniform over RES_CHOICES (optionally scaled down for tests),
    magnification log-uniform in [1, 64], filter bilinear or B-spline with probability 1/2 each,
    a random window origin inside the texture; shading with the 8-channel layout."""
    rng = np.random.default_rng(seed)
    views = []
    for i in range(n):
        w, h = RES_CHOICES[int(rng.integers(0, len(RES_CHOICES)))]
        w, h = max(8, int(round(w * scale / 8)) * 8), max(4, int(round(h * scale / 4)) * 4)
        mag = float(np.exp(rng.uniform(0.0, math.log(64.0))))
        filt = int(rng.integers(0, 2))
        span_x, span_y = w / mag, h / mag
        ox = float(rng.uniform(0.0, max(0.0, tex - span_x)))
        oy = float(rng.uniform(0.0, max(0.0, tex - span_y)))
        v = screen_aligned_view(w, h, tex, tex, mag, filt, origin=(ox, oy), view_id=i)
        v = with_shading(v, "c3")
        v["magnification"] = mag
        views.append(v)
    return views
