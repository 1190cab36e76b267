"""CPU oracle of the learned initial guess and of spectral upsampling -- TEST
INFRASTRUCTURE ONLY (imported by tests/ and nothing in the product path).

Plain numpy forward and backward of the guess network, layer by layer, with
no fusion.  With ``bf16=True`` every GEMM operand is rounded to bfloat16
(round to nearest even) before an FP64 product, and every layer output is
stored as float32, which is the arithmetic contract of the CUDA kernels
(BF16 operands, FP32 accumulation and storage); with ``bf16=False`` it is the
exact FP64 network, which the finite-difference pins check.

Network (parameters are one flat float32 vector, in this order):
  W1 (16 x 256, rows 8..15 zero padding), b1 (256), W2 (256 x 8192), b2 (8192),
  W3 (32 x 128), b3 (16), W4 (16 x 64), b4 (8), W5 (8 x 8), b5 (2).
  h1 = relu(f W1 + b1); z = h1 W2 + b2 (latent: 256 voxels of a 4x8x8 grid x
  32 channels, voxel-major); y1 = relu(z_vox W3 + b3[col % 16]);
  y2 = relu(y1_vox W4 + b4[col % 8]); o = y2_vox W5 + b5[col % 2];
  each "_vox" view is the previous output with rows = voxels; output columns
  are (sub-position, channel) of a transposed convolution whose kernel equals
  its stride.  The loss per sample is 1 - |<u,t>|^2 / (|u|^2 |t|^2).
"""
from __future__ import annotations

import numpy as np

from .atkm_oracle import spectral_upsample  # noqa: F401  (re-exported for the guess tests)

F, FPAD, H, Z, C0, V0 = 8, 16, 256, 8192, 32, 256
C1, C2, C3 = 16, 8, 2
N1, N2, N3 = 8 * C1, 8 * C2, 4 * C3
OUT = (16, 64, 64)

SHAPES = [("W1", (FPAD, H)), ("b1", (H,)), ("W2", (H, Z)), ("b2", (Z,)), ("W3", (C0, N1)), ("b3", (C1,)),
          ("W4", (C1, N2)), ("b4", (C2,)), ("W5", (C2, N3)), ("b5", (C3,))]
NUM_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16_round(x) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest, ties to even), as float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def unpack(params, dtype=np.float32) -> dict:
    p = np.asarray(params, dtype=dtype)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def _mm(a, b, bf16):
    """a @ b with the kernels' operand rounding (bf16) or exactly (FP64)."""
    if bf16:
        return bf16_round(a).astype(np.float64) @ bf16_round(b).astype(np.float64)
    return np.asarray(a, np.float64) @ np.asarray(b, np.float64)


def _store(x, bf16):
    return x.astype(np.float32) if bf16 else x


def _bias(x, b, cb, bf16):
    cols = x.shape[1]
    bb = np.tile(np.asarray(b)[:cb], cols // cb)
    if bf16:
        return (x.astype(np.float32) + bb.astype(np.float32)).astype(np.float32)
    return x + bb


def pad_features(feats) -> np.ndarray:
    f = np.asarray(feats, dtype=np.float32)
    out = np.zeros((f.shape[0], FPAD), dtype=np.float32)
    out[:, :F] = f
    return out


def forward(params, feats, bf16=True) -> dict:
    P = unpack(params, np.float32 if bf16 else np.float64)
    B = feats.shape[0]
    f = pad_features(feats) if bf16 else np.concatenate([np.asarray(feats, np.float64),
                                                         np.zeros((B, FPAD - F))], axis=1)
    h1 = np.maximum(_bias(_store(_mm(f, P["W1"], bf16), bf16), P["b1"], H, bf16), 0)
    z = _bias(_store(_mm(h1, P["W2"], bf16), bf16), P["b2"], Z, bf16)
    zv = z.reshape(B * V0, C0)
    y1 = np.maximum(_bias(_store(_mm(zv, P["W3"], bf16), bf16), P["b3"], C1, bf16), 0)
    y1v = y1.reshape(B * V0 * 8, C1)
    y2 = np.maximum(_bias(_store(_mm(y1v, P["W4"], bf16), bf16), P["b4"], C2, bf16), 0)
    y2v = y2.reshape(B * V0 * 64, C2)
    o = _bias(_store(_mm(y2v, P["W5"], bf16), bf16), P["b5"], C3, bf16)
    return dict(f=f, h1=h1, z=z, zv=zv, y1=y1, y1v=y1v, y2=y2, y2v=y2v, o=o, B=B)


def out_index(B):
    """Grid coordinates (b, z, y, x, ch) of every element of the L3 output."""
    rows = np.arange(B * V0 * 64)
    s2 = rows & 7
    s1 = (rows >> 3) & 7
    r0 = rows >> 6
    v0 = r0 % V0
    b = r0 // V0
    iz, iy, ix = v0 >> 6, (v0 >> 3) & 7, v0 & 7
    cols = np.arange(N3)
    ch = cols & 1
    s3 = cols >> 1
    z = ((iz * 2 + (s1 >> 2)) * 2 + (s2 >> 2))[:, None] + 0 * cols[None, :]
    y = ((((iy * 2 + ((s1 >> 1) & 1)) * 2 + ((s2 >> 1) & 1)) * 2)[:, None] + (s3 >> 1)[None, :])
    x = ((((ix * 2 + (s1 & 1)) * 2 + (s2 & 1)) * 2)[:, None] + (s3 & 1)[None, :])
    bb = b[:, None] + 0 * cols[None, :]
    return bb, z, y, x, np.broadcast_to(ch[None, :], z.shape)


def out_to_psi(o, B) -> np.ndarray:
    bb, z, y, x, ch = out_index(B)
    psi = np.zeros((B,) + OUT, dtype=np.complex128)
    re = ch == 0
    psi[bb[re], z[re], y[re], x[re]] += o[re]
    psi[bb[~re], z[~re], y[~re], x[~re]] += 1j * o[~re]
    return psi


def loss_and_grad(params, feats, targets, bf16=True):
    """Batch-mean loss and its gradient w.r.t. the flat parameter vector."""
    P = unpack(params, np.float32 if bf16 else np.float64)
    a = forward(params, feats, bf16)
    B = a["B"]
    u = out_to_psi(a["o"], B)
    t = np.asarray(targets, dtype=np.complex128)
    s = np.sum(u * np.conj(t), axis=(1, 2, 3))
    uu = np.sum(np.abs(u) ** 2, axis=(1, 2, 3))
    tt = np.sum(np.abs(t) ** 2, axis=(1, 2, 3))
    loss = float(np.mean(1.0 - np.abs(s) ** 2 / (uu * tt)))
    # dL/d(Re u) + i dL/d(Im u)
    g = -2.0 / B * (s[:, None, None, None] * t / (uu * tt)[:, None, None, None]
                    - (np.abs(s) ** 2 / (uu ** 2 * tt))[:, None, None, None] * u)
    bb, z, y, x, ch = out_index(B)
    gv = g[bb, z, y, x]
    dO = np.where(ch == 0, gv.real, gv.imag)
    dO = _store(dO, bf16)
    G = {}
    # L3
    G["W5"] = _mm(a["y2v"].T, dO, bf16)
    G["b5"] = dO.reshape(-1, N3 // C3, C3).sum(axis=(0, 1))
    dy2 = _store(_mm(dO, P["W5"].T, bf16), bf16).reshape(B * V0 * 8, N2)
    dy2 = np.where(a["y2"] > 0, dy2, 0)
    # L2
    G["W4"] = _mm(a["y1v"].T, dy2, bf16)
    G["b4"] = dy2.reshape(-1, N2 // C2, C2).sum(axis=(0, 1))
    dy1 = _store(_mm(dy2, P["W4"].T, bf16), bf16).reshape(B * V0, N1)
    dy1 = np.where(a["y1"] > 0, dy1, 0)
    # L1
    G["W3"] = _mm(a["zv"].T, dy1, bf16)
    G["b3"] = dy1.reshape(-1, N1 // C1, C1).sum(axis=(0, 1))
    dz = _store(_mm(dy1, P["W3"].T, bf16), bf16).reshape(B, Z)
    # MLP2
    G["W2"] = _mm(a["h1"].T, dz, bf16)
    G["b2"] = dz.sum(axis=0)
    dh1 = _store(_mm(dz, P["W2"].T, bf16), bf16)
    dh1 = np.where(a["h1"] > 0, dh1, 0)
    # MLP1
    G["W1"] = _mm(a["f"].T, dh1, bf16)
    G["b1"] = dh1.sum(axis=0)
    return loss, pack(G)


def loss(params, feats, targets, bf16=True) -> float:
    """Batch-mean loss only (forward pass and the loss formula)."""
    a = forward(params, feats, bf16)
    u = out_to_psi(a["o"], a["B"])
    t = np.asarray(targets, dtype=np.complex128)
    s = np.sum(u * np.conj(t), axis=(1, 2, 3))
    uu = np.sum(np.abs(u) ** 2, axis=(1, 2, 3))
    tt = np.sum(np.abs(t) ** 2, axis=(1, 2, 3))
    return float(np.mean(1.0 - np.abs(s) ** 2 / (uu * tt)))
