"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only: no projection, product or
correlation arithmetic of the method.  Both the CUDA path (tests, bench) and
the CPU oracle read the same arrays from here, so the two see identical bits.

All draws use numpy's PCG64 ``default_rng(seed)``.  The recipes stand in for
data the paper used but that is not available here: the image/audio inputs
normalised to [-1, 1] of Sec. IV, the Yale face images of Sec. V-A and the
cover-song beat/tempo features of Sec. V-B.
"""
from __future__ import annotations

import os

import numpy as np

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_cache")


def uniform_pair(M: int = 256, K: int = 512, N: int = 256, seed: int = 0):
    """A (M x K) then B (K x N), i.i.d. uniform[-1, 1) from one stream, float64."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1.0, 1.0, size=(M, K))
    B = rng.uniform(-1.0, 1.0, size=(K, N))
    return A, B


def audio_signal(S: int = 1 << 20, n_tones: int = 32, fs: float = 44100.0,
                 f_lo: float = 50.0, f_hi: float = 8000.0, snr_db: float = 20.0,
                 seed: int = 0, rng=None) -> np.ndarray:
    """Sum of sinusoids with random frequencies plus white Gaussian noise.

    f_i ~ U[f_lo, f_hi] Hz at sampling rate fs, amplitudes ~ U[0.1, 1],
    phases ~ U[0, 2 pi); noise variance = signal power / 10^(snr_db/10).
    Returned as float32 (the CONV workload's input precision).
    """
    if rng is None:
        rng = np.random.default_rng(seed)
    f = rng.uniform(f_lo, f_hi, size=n_tones)
    a = rng.uniform(0.1, 1.0, size=n_tones)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n_tones)
    n = np.arange(S, dtype=np.float64)
    x = np.zeros(S, dtype=np.float64)
    for i in range(n_tones):
        x += a[i] * np.sin(2.0 * np.pi * f[i] / fs * n + ph[i])
    p_sig = float(np.mean(x * x))
    x += rng.normal(0.0, np.sqrt(p_sig / 10.0 ** (snr_db / 10.0)), size=S)
    return x.astype(np.float32)


def audio_workload(S: int = 1 << 20, T: int = 4096, n_templates: int = 64, seed: int = 0,
                   **kw):
    """One audio-like signal and n_templates windows of length T cut from it.

    Template offsets are uniform over [0, S - T], so every template has an
    exact match somewhere in the signal.  Returns (signal[S], templates[nt, T],
    offsets[nt]) with float32 data.
    """
    rng = np.random.default_rng(seed)
    s = audio_signal(S, seed=seed, rng=rng, **kw)
    off = rng.integers(0, S - T + 1, size=n_templates)
    k = np.stack([s[o:o + T] for o in off]).astype(np.float32)
    return s, k, off


def _blur_fields(n: int, h: int, w: int, sigma: float, rng) -> np.ndarray:
    """n white-noise fields of h x w, Gaussian-blurred (periodic, via FFT)."""
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.rfftfreq(w)[None, :]
    H = np.exp(-2.0 * (np.pi * sigma) ** 2 * (fx * fx + fy * fy))
    out = np.empty((n, h, w), dtype=np.float64)
    step = 256
    for i in range(0, n, step):
        z = rng.standard_normal((min(step, n - i), h, w))
        out[i:i + step] = np.fft.irfft2(np.fft.rfft2(z) * H, s=(h, w))
    return out


def face_probes(n: int = 4096, h: int = 92, w: int = 112, sigma: float = 4.0,
                seed: int = 0) -> np.ndarray:
    """Face-image stand-ins: smooth random fields quantised to 8-bit grey levels.

    Each field is min-max scaled to [0, 1], rounded to k/255 and flattened
    row-major to h*w values.  Returned as float32, shape (n, h*w).
    """
    rng = np.random.default_rng(seed)
    f = _blur_fields(n, h, w, sigma, rng)
    lo = f.min(axis=(1, 2), keepdims=True)
    hi = f.max(axis=(1, 2), keepdims=True)
    f = (f - lo) / (hi - lo)
    f = np.round(255.0 * f) / 255.0
    return f.reshape(n, h * w).astype(np.float32)


def orthonormal_features(K: int = 10304, N: int = 2048, seed: int = 1,
                         cache: bool = True) -> np.ndarray:
    """K x N feature matrix with orthonormal columns (QR of a Gaussian matrix), float32."""
    path = os.path.join(_CACHE, f"orthofeat_{K}x{N}_s{seed}.npy")
    if cache and os.path.exists(path):
        return np.load(path)
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((K, N))
    Q, Rr = np.linalg.qr(G)
    Q *= np.sign(np.diag(Rr))[None, :]
    Q = Q.astype(np.float32)
    if cache:
        os.makedirs(_CACHE, exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp.npy"
        np.save(tmp, Q)
        os.replace(tmp, path)
    return Q


def gaussian(shape, std: float = 1.0, seed: int = 0) -> np.ndarray:
    """i.i.d. N(0, std^2) float32 array."""
    rng = np.random.default_rng(seed)
    return (std * rng.standard_normal(shape)).astype(np.float32)


def layer_workload(M: int = 8192, K: int = 4096, N: int = 4096, std: float = 0.02,
                   seed: int = 1):
    """X (M x K), W (K x N) ~ N(0, std^2) and upstream gradient dY (M x N) ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    X = (std * rng.standard_normal((M, K))).astype(np.float32)
    W = (std * rng.standard_normal((K, N))).astype(np.float32)
    dY = rng.standard_normal((M, N)).astype(np.float32)
    return X, W, dY


def uneven_batch_sizes(n_gemm: int = 512, n_conv: int = 256, seed: int = 0):
    """Sizes of the uneven batch: GEMMs with M, N ~ U{64..2048}, K ~ U{256..8192};
    correlations with S ~ U{2^14..2^20} and one template of 1024."""
    rng = np.random.default_rng(seed)
    gemms = [(int(rng.integers(64, 2049)), int(rng.integers(64, 2049)), int(rng.integers(256, 8193)))
             for _ in range(n_gemm)]
    convs = [int(rng.integers(1 << 14, (1 << 20) + 1)) for _ in range(n_conv)]
    return gemms, convs


def device_normal(shape, seed: int, device, dtype=None):
    """N(0, 1) tensor drawn on a CUDA device from a seeded counter-based generator (Philox)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    x = torch.randn(shape, generator=g, device=device, dtype=torch.float32)
    return x if dtype is None else x.to(dtype)
