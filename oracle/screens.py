"""Von Karman phase screens by the FFT method with subharmonics (FP64).

Follows AtmoEvolution (App. A, Tab. 4: "turbulence model based on finite phase
screens") with the parameters of App. B, Listing 2 (``L0``, ``Cn2``, ``seed``).
The paper gives no formula; this is the textbook construction:

* Phase power spectrum at 500 nm, in rad^2 m^2:
      Phi(f) = 0.023 r0^(-5/3) (|f|^2 + L0^-2)^(-11/6),   Phi(0) = 0
  (L0 = inf gives Kolmogorov).
* On an M x M grid of pitch Delta, frequency samples f_k = k_fft / (M Delta)
  with k_fft the signed FFT index (0..M/2-1, -M/2..-1); df = 1 / (M Delta).
      screen[y, x] = Re sum_k c_k sqrt(Phi(f_k)) df exp(2 pi i f_k . (x, y) Delta)
  with c_k complex noise whose real and imaginary parts are standard normal.
* Subharmonics: levels p = 1..3 with spacing df / 3^p, the eight offsets
  (a, b) in {-1, 0, 1}^2 minus (0, 0), same amplitude rule with df -> df_p;
  their sum has its mean over the screen removed.

Both noise sets are inputs (drawn by ``synth``).
"""
import math

import numpy as np


def vk_psd(fx, fy, r0: float, L0: float):
    """Phi(f) in rad^2 m^2 at the wavelength r0 refers to (500 nm)."""
    f2 = np.asarray(fx, dtype=np.float64) ** 2 + np.asarray(fy, np.float64) ** 2
    k0 = 0.0 if math.isinf(L0) else 1.0 / (L0 * L0)
    base = f2 + k0
    out = np.zeros_like(base)
    nz = f2 > 0          # Phi(0) = 0: the piston sample carries no power
    out[nz] = 0.023 * r0 ** (-5.0 / 3.0) * base[nz] ** (-11.0 / 6.0)
    return out


def fft_freqs(M: int, delta: float) -> np.ndarray:
    """Signed FFT frequency of each index: k / (M delta), k >= M/2 wrapped."""
    k = np.arange(M, dtype=np.int64)
    k = np.where(k >= M // 2, k - M, k)
    return k.astype(np.float64) / (M * delta)


def fft_screen(M: int, delta: float, r0: float, L0: float,
               cn: np.ndarray, cn_sub: np.ndarray) -> np.ndarray:
    """(M, M) float64 phase screen [rad at 500 nm]; row = y, column = x."""
    df = 1.0 / (M * delta)
    f = fft_freqs(M, delta)
    amp = np.sqrt(vk_psd(f[None, :], f[:, None], r0, L0)) * df
    # sum_k a_k exp(+2 pi i k n / M) == M^2 * ifft2(a)
    scr = np.real(np.fft.ifft2(cn * amp)) * (M * M)

    pos = np.arange(M, dtype=np.float64) * delta
    sub = np.zeros((M, M))
    for p in range(1, cn_sub.shape[0] + 1):
        dfp = df / 3.0 ** p
        for b in range(3):
            for a in range(3):
                if a == 1 and b == 1:
                    continue
                fx = (a - 1) * dfp
                fy = (b - 1) * dfp
                ap = math.sqrt(float(vk_psd(np.array(fx), np.array(fy), r0, L0))) * dfp
                ex = np.exp(2j * math.pi * fx * pos)
                ey = np.exp(2j * math.pi * fy * pos)
                sub += np.real(cn_sub[p - 1, b, a] * ap * ey[:, None] * ex[None, :])
    sub -= sub.mean()
    return scr + sub


def expected_structure_function(M: int, delta: float, r0: float, L0: float,
                                r_px: np.ndarray, levels: int = 3) -> np.ndarray:
    """Exact ensemble mean of (phi(x + r) - phi(x))^2 for separations of r_px
    pixels along x, for the generator above:
        E[D(r)] = sum over all frequency samples of 2 a_k^2 (1 - cos 2 pi f_x r)
    (each sample contributes independently; E|Re(c e^{i t})|^2 = 1)."""
    df = 1.0 / (M * delta)
    f = fft_freqs(M, delta)
    a2 = vk_psd(f[None, :], f[:, None], r0, L0) * df * df
    out = []
    for r in np.atleast_1d(r_px):
        rm = r * delta
        d = 2.0 * np.sum(a2 * (1.0 - np.cos(2 * math.pi * f[None, :] * rm)))
        for p in range(1, levels + 1):
            dfp = df / 3.0 ** p
            for b in range(3):
                for a in range(3):
                    if a == 1 and b == 1:
                        continue
                    fx, fy = (a - 1) * dfp, (b - 1) * dfp
                    ap2 = float(vk_psd(np.array(fx), np.array(fy), r0, L0)) * dfp * dfp
                    d += 2.0 * ap2 * (1.0 - math.cos(2 * math.pi * fx * rm))
        out.append(d)
    return np.array(out)


def kolmogorov_structure_function(r_m, r0: float):
    """D(r) = 6.88 (r / r0)^(5/3) rad^2."""
    return 6.88 * (np.asarray(r_m, dtype=np.float64) / r0) ** (5.0 / 3.0)
