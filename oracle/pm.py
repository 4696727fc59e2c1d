"""FP64 CPU oracle for the long-range (PM) part of the force split and the KDK step.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: imported by the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg, never by the
product package.

Force split (Sec. 2.2): the pair potential 1/r = erfc(r/2r_s)/r + erf(r/2r_s)/r.
The short-range part is the truncated FMM; the long-range part is the periodic
convolution of the mass density with erf(r/2r_s)/r, whose Fourier transform is
4 pi exp(-k^2 r_s^2) / k^2, evaluated on the PM mesh (Sec. 2.2):
  1. cloud-in-cell (CIC) mass assignment to the mesh points x_g = g L / N_g,
  2. FFT of the mass mesh,
  3. a(k) = i k G 4 pi exp(-k^2 r_s^2) / k^2 / W(k)^2 * m(k) / L^3 with
     W(k) = prod_d sinc^2(k_d L / 2 N_g) (the CIC window, divided out once for
     the assignment and once for the interpolation); the k = 0 mode and the
     Nyquist plane of each gradient component are zero,
  4. inverse FFT of each component and CIC interpolation to the particles.
Sign: a = G grad Phi with Phi = sum_j m_j psi(x - x_j), the convention of the
short-range pair force a_i = G sum_j m_j f_(1)(r) r (attractive, f_(1) < 0).

The time step (the synchronised global step of Sec. 4) is the kick-drift-kick
leapfrog in static space:
  v += a dt/2;  x += v dt (wrapped into the box);  a = a_SR + a_LR at the new x;  v += a dt/2.

Parity status: pinned by closed forms in tests/test_oracle_pm.py (a plane-wave
mass field on the mesh points, the spectral sum of the periodic long-range pair
force, momentum conservation, and short + long range = Newtonian).
"""
from __future__ import annotations

import numpy as np


def _cic(pos, box, ng):
    """Mesh index of the lower corner and the weights along each axis (FP64)."""
    u = np.asarray(pos, dtype=np.float64) / box * ng  # [3][n], mesh units
    u = np.mod(u, ng)
    i0 = np.floor(u).astype(np.int64)
    d = u - i0
    i0 = np.mod(i0, ng)
    return i0, d


def cic_deposit(pos, mass, box, ng):
    """Mass per mesh point, [ng][ng][ng] (index order x, y, z)."""
    i0, d = _cic(pos, box, ng)
    rho = np.zeros((ng, ng, ng))
    mass = np.asarray(mass, dtype=np.float64)
    for ox in (0, 1):
        wx = d[0] if ox else 1.0 - d[0]
        for oy in (0, 1):
            wy = d[1] if oy else 1.0 - d[1]
            for oz in (0, 1):
                wz = d[2] if oz else 1.0 - d[2]
                np.add.at(rho, ((i0[0] + ox) % ng, (i0[1] + oy) % ng, (i0[2] + oz) % ng), mass * wx * wy * wz)
    return rho


def cic_interpolate(field, pos, box):
    """Values of a mesh field [ng][ng][ng] at the particles by CIC weights."""
    ng = field.shape[0]
    i0, d = _cic(pos, box, ng)
    out = np.zeros(i0.shape[1])
    for ox in (0, 1):
        wx = d[0] if ox else 1.0 - d[0]
        for oy in (0, 1):
            wy = d[1] if oy else 1.0 - d[1]
            for oz in (0, 1):
                wz = d[2] if oz else 1.0 - d[2]
                out += wx * wy * wz * field[(i0[0] + ox) % ng, (i0[1] + oy) % ng, (i0[2] + oz) % ng]
    return out


def wavenumbers(ng, box):
    """k along one axis for the full (n) and the half (rfft) index ranges."""
    n = np.arange(ng)
    kfull = 2.0 * np.pi / box * np.where(n <= ng // 2, n, n - ng)
    khalf = 2.0 * np.pi / box * np.arange(ng // 2 + 1)
    return kfull, khalf


def long_range_mesh(rho, box, rs, G=1.0, green_k2=None):
    """Long-range acceleration on the mesh points, [3][ng][ng][ng], from the mass mesh.
    green_k2 (optional): the long-range Green function of another split as a
    function of k^2 > 0 (default: the Gaussian 4 pi exp(-k^2 r_s^2) / k^2)."""
    ng = rho.shape[0]
    mk = np.fft.rfftn(rho)
    kf, kh = wavenumbers(ng, box)
    kx = kf[:, None, None]
    ky = kf[None, :, None]
    kz = kh[None, None, :]
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    h = box / ng

    def sinc(x):
        return np.sinc(x / np.pi)  # sin(x) / x

    w = (sinc(kx * h / 2) * sinc(ky * h / 2) * sinc(kz * h / 2)) ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        if green_k2 is None:
            green = np.where(k2 > 0, 4.0 * np.pi * G * np.exp(-k2 * rs ** 2) / k2 / w ** 2, 0.0)
        else:
            kk = np.where(k2 > 0, k2, 1.0)
            green = np.where(k2 > 0, G * np.asarray(green_k2(kk.ravel())).reshape(k2.shape) / w ** 2, 0.0)
    phi = green * mk / box ** 3
    nyq = ng // 2 if ng % 2 == 0 else -1
    out = np.zeros((3, ng, ng, ng))
    for d, kd in enumerate((kx, ky, kz)):
        kd = np.broadcast_to(kd, k2.shape).copy()
        if nyq >= 0:
            if d < 2:
                sl = [slice(None)] * 3
                sl[d] = nyq
                kd[tuple(sl)] = 0.0
            else:
                kd[:, :, nyq] = 0.0
        # numpy's inverse FFT divides by ng^3; the Fourier series sums the modes
        out[d] = np.fft.irfftn(1j * kd * phi, s=(ng, ng, ng), axes=(0, 1, 2)) * ng ** 3
    return out


def pm_long_range(pos, mass, box, ng, rs, G=1.0, green_k2=None):
    """Long-range accelerations [3][n] of the particles (FP64); green_k2 as in long_range_mesh."""
    rho = cic_deposit(pos, mass, box, ng)
    a = long_range_mesh(rho, box, rs, G, green_k2)
    return np.stack([cic_interpolate(a[d], pos, box) for d in range(3)])


def lr_pair_spectral(r_vec, m, box, rs, G=1.0, kmax_rs=7.0):
    """Periodic long-range acceleration at displacement r_vec from a point mass m,
    by direct summation of the Fourier series (no mesh):
        a(r) = G m / L^3 sum_{k != 0} 4 pi exp(-k^2 r_s^2) / k^2 * i k exp(i k.r)
             = -G m / L^3 sum_{k != 0} 4 pi exp(-k^2 r_s^2) / k^2 * k sin(k.r)."""
    nmax = int(np.ceil(kmax_rs / rs * box / (2 * np.pi)))
    n = np.arange(-nmax, nmax + 1)
    kx, ky, kz = np.meshgrid(n, n, n, indexing="ij")
    k = 2 * np.pi / box * np.stack([kx.ravel(), ky.ravel(), kz.ravel()])
    k2 = (k ** 2).sum(0)
    sel = k2 > 0
    k, k2 = k[:, sel], k2[sel]
    amp = 4 * np.pi * np.exp(-k2 * rs ** 2) / k2
    s = np.sin(k.T @ np.asarray(r_vec, dtype=np.float64))
    return -G * m / box ** 3 * (k * (amp * s)).sum(axis=1)


def kdk_step(pos, vel, acc, dt, box, forces):
    """One kick-drift-kick step; ``forces(pos) -> acc`` gives the total acceleration."""
    vel = vel + 0.5 * dt * acc
    pos = np.mod(pos + dt * vel, box)
    acc = forces(pos)
    vel = vel + 0.5 * dt * acc
    return pos, vel, acc
