"""FP64 CPU oracle for the confined Toner-Tu-Swift-Hohenberg (TTSH) vorticity solver.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or executes this
module: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may use it.  It shares no code with the CUDA path; the only module both sides
use is ``ttsh_inputs`` (seeded masks and noise, none of the method's arithmetic).

What it computes, in the paper's order and notation, all in float64:

* the unitary DFT of Appendix D: f^(k) = N^-1 sum_x f(x) e^{-i k.x}, inverse with e^{+i k.x}
  and the same N^-1 (``dft2`` / ``idft2`` via numpy's pocketfft with norm="ortho";
  ``dft2_naive`` / ``idft2_naive`` write the definition out as dense matrices);
* Algorithm 2 (Appendix E, mask processing): K = (iDFT[ lowpass_{1/4}( DFT[K_naive] ) ])^2;
* Algorithm 1 (Appendix D, integration scheme): one pseudospectral integrating-factor Euler
  step of Eq. (mod2), with the k = 0 mean-flow update of Eq. (avg), the 1/2-rule dealiasing,
  the Hermitian projection and the stream-function velocity recovery;
* diagnostics: energy, enstrophy, the vortex order parameter Psi (Sec. III.C) and the shell
  spectrum E(s).

Readings where the paper is silent or inconsistent (also listed in the design notes):
* c1  nabla <-> +ik, consistent with the DFT sign above and with Algorithm 1 (the prose says
  "-ik"; that would contradict Algorithm 1's own +ik and the stream function relations);
* c2  the 1/2 rule keeps integer index radius |m|^2 <= (N/4)^2, k = dk*m, dk = 2 pi/(N dx);
* c3  the 1/4 mask cutoff keeps |m|^2 <= (N/8)^2;
* c7  omega = Re iDFT[omega^] (real by the Hermitian invariant), and likewise every field
  brought to real space is the real part of its inverse transform;
* c6  the initial state is the projection of a real velocity field (``project_velocity``);
* c11 energy E = (2N^2)^-1 sum_x |v|^2, enstrophy Z = (2N^2)^-1 sum_x omega^2, shell spectrum
  E(s) = (2N^2)^-1 sum_{round|m| = s} |v^(m)|^2, mean-flow = v^(0)/N;
* c12 Psi sums over every grid point, e_theta(centre) := 0.

Every function cites the passage it follows.  There is no blocking, fusion or reordering
beyond what the scheme of Appendix D states.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np


@dataclass(frozen=True)
class Params:
    """Model and discretisation constants (Table I).  n: grid points per side."""
    n: int
    dx: float
    a: float = 0.5
    b: float = 1.6
    lam: float = 9.0
    gamma_v: float = 40.0
    gamma_w: float = 4.0
    dt: float = 0.01

    def with_(self, **kw) -> "Params":
        return replace(self, **kw)


@dataclass
class State:
    """The scheme's state at time t: real velocity v and vorticity spectrum omega^."""
    vx: np.ndarray      # real (n, n), indexed [y][x]
    vy: np.ndarray      # real (n, n)
    w_hat: np.ndarray   # complex (n, n), FFT order, indexed [ky][kx]

    def copy(self) -> "State":
        return State(self.vx.copy(), self.vy.copy(), self.w_hat.copy())


# ----------------------------------------------------------------------------------------
# DFT of Appendix D (unitary, 1/sqrt(N^2) both ways)
# ----------------------------------------------------------------------------------------

def dft2(f: np.ndarray) -> np.ndarray:
    """f^(k) = N^-1 sum_x f(x) exp(-i k.x) (Appendix D), via pocketfft."""
    return np.fft.fft2(f, norm="ortho")


def idft2(F: np.ndarray) -> np.ndarray:
    """f(x) = N^-1 sum_k f^(k) exp(+i k.x) (Appendix D), via pocketfft."""
    return np.fft.ifft2(F, norm="ortho")


def threaded_dft(workers: int | None = None):
    """The same unitary DFT pair computed by scipy.fft on `workers` threads (default: every
    host core) - a library primitive like numpy's pocketfft, for running the oracle at large
    grid sizes in tests.  Returns (dft, idft) to pass to the functions below."""
    import os

    import scipy.fft as sf
    w = workers or os.cpu_count() or 1

    def dft(f):
        return sf.fft2(f, norm="ortho", workers=w)

    def idft(F):
        return sf.ifft2(F, norm="ortho", workers=w)

    return dft, idft


def _dft_matrix(n: int, sign: int) -> np.ndarray:
    j = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(j, j) / n)


def dft2_naive(f: np.ndarray) -> np.ndarray:
    """The same unitary DFT written out as the separable double sum (dense matrices)."""
    n = f.shape[0]
    E = _dft_matrix(n, -1)
    return (E @ f @ E.T) / n


def idft2_naive(F: np.ndarray) -> np.ndarray:
    n = F.shape[0]
    E = _dft_matrix(n, +1)
    return (E @ F @ E.T) / n


# ----------------------------------------------------------------------------------------
# Wavenumber grid (Table I: k in [-pi/dx, pi/dx]^2, dk = 2 pi / L, L = N dx)
# ----------------------------------------------------------------------------------------

def index_grid(n: int):
    """Integer mode indices (mx, my), each (n, n) in FFT order, indexed [ky][kx]."""
    m = np.fft.fftfreq(n, d=1.0 / n).astype(np.int64)
    MX, MY = np.meshgrid(m, m, indexing="xy")
    return MX, MY


def wavenumbers(p: Params):
    dk = 2.0 * np.pi / (p.n * p.dx)
    MX, MY = index_grid(p.n)
    return dk * MX, dk * MY, MX * MX + MY * MY


def mirror(F: np.ndarray) -> np.ndarray:
    """F(-k) in FFT order: index j -> (-j) mod n on both axes."""
    return np.roll(np.flip(F, axis=(0, 1)), shift=1, axis=(0, 1))


# ----------------------------------------------------------------------------------------
# Algorithm 2 (Appendix E): mask processing
# ----------------------------------------------------------------------------------------

def process_mask(k_naive: np.ndarray, dft=dft2, idft=idft2) -> np.ndarray:
    """K = (iDFT[K^_naive with |k|^2 > (pi/(4 dx))^2 set to 0])^2; no optional filtering.

    The cutoff pi/(4 dx) equals dk * N/8, so the integer test is |m|^2 > (N/8)^2 (reading c3).
    """
    n = k_naive.shape[0]
    K_hat = dft(k_naive.astype(np.float64))
    MX, MY = index_grid(n)
    K_hat = np.where(MX * MX + MY * MY > (n // 8) ** 2, 0.0, K_hat)
    return np.real(idft(K_hat)) ** 2


# ----------------------------------------------------------------------------------------
# Algorithm 1 (Appendix D): one integration step
# ----------------------------------------------------------------------------------------

def _post_process(w_naive, v0_new, p: Params):
    """Projection that ends every step (Appendix D): omega^(0) = 0 with the mean flow v^(0)
    from Eq. (avg), removal of the modes beyond the 1/2 rule, the Hermitian average, and the
    velocity from the stream function, psi^ = omega^/k^2, v^ = (i ky psi^, -i kx psi^).

    Returns (omega^_new, v^x_new, v^y_new) on the full FFT-ordered grid.
    """
    n = p.n
    KX, KY, M2 = wavenumbers(p)
    is_zero = M2 == 0
    aliased = M2 > (n // 4) ** 2           # k^2 > (pi/(2 dx))^2  <=>  |m|^2 > (N/4)^2
    keep = ~is_zero & ~aliased

    w_new = np.zeros_like(w_naive)
    vx_new = np.zeros_like(w_naive)
    vy_new = np.zeros_like(w_naive)
    # k = 0: omega^ = 0, v^(0) from the space-averaged equation (passed in).
    vx_new[0, 0] = v0_new[0]
    vy_new[0, 0] = v0_new[1]
    # 0 < k^2 <= cutoff: Hermitian average, psi^ = omega^/k^2, v^ = (i ky psi^, -i kx psi^).
    herm = 0.5 * (w_naive + np.conj(mirror(w_naive)))
    w_new[keep] = herm[keep]
    k2 = KX * KX + KY * KY
    psi = np.zeros_like(w_naive)
    psi[keep] = w_new[keep] / k2[keep]
    vx_new[keep] = 1j * KY[keep] * psi[keep]
    vy_new[keep] = -1j * KX[keep] * psi[keep]
    return w_new, vx_new, vy_new


def linear_rate(k2: np.ndarray, p: Params) -> np.ndarray:
    """Growth rate of the linear part of Eq. (mod2) at |k|^2 = k2: a - (1 - k^2)^2 (the
    Swift-Hohenberg operator a - (1 + nabla^2)^2 in Fourier space)."""
    return p.a - (1.0 - k2) ** 2


def nonlinear_terms(vx, vy, omega, gx, gy, K, p: Params):
    """The non-linear and mask terms of Eq. (mod2) in real space, before the curl.

    Velocity-level part (its curl enters the vorticity equation; Sec. II.A):
        f_v = -b |v|^2 v - gamma_v K v
    Vorticity-level part, with grad(omega) = (gx, gy):
        f_w = -lambda v . grad(omega) - gamma_w K omega
    """
    v2 = vx * vx + vy * vy
    fvx = -p.b * v2 * vx - p.gamma_v * K * vx
    fvy = -p.b * v2 * vy - p.gamma_v * K * vy
    fw = -p.lam * (vx * gx + vy * gy) - p.gamma_w * K * omega
    return fvx, fvy, fw


def step(s: State, K: np.ndarray, p: Params, dft=dft2, idft=idft2) -> State:
    """One time step of Eq. (mod2) with the pseudospectral integrating-factor Euler scheme of
    Appendix D: the linear operator is integrated exactly over dt, the non-linear and mask
    terms by forward Euler, then the k = 0 mean flow follows the space-averaged equation
    Eq. (avg) and the spectrum is projected (Hermitian, 1/2 rule, stream-function velocity).
    Returns (v(t+dt), omega^(t+dt))."""
    KX, KY, _ = wavenumbers(p)
    vx, vy, w_hat = s.vx, s.vy, s.w_hat
    # real-space fields the non-linear terms need; nabla <-> +ik (reading c1), real parts
    # (reading c7)
    omega = np.real(idft(w_hat))
    gx = np.real(idft(1j * KX * w_hat))
    gy = np.real(idft(1j * KY * w_hat))
    fvx, fvy, fw = nonlinear_terms(vx, vy, omega, gx, gy, K, p)
    # Fourier transform of the vorticity equation's non-linear part: the z-component of the
    # curl of f_v, i(kx f^_vy - ky f^_vx), plus f^_w
    Fvx, Fvy, Fw = dft(fvx), dft(fvy), dft(fw)
    n_hat = 1j * (KX * Fvy - KY * Fvx) + Fw
    # integrating-factor Euler: omega^ <- exp(L(k) dt) (omega^ + dt N^(k))
    k2 = KX * KX + KY * KY
    w_naive = np.exp(linear_rate(k2, p) * p.dt) * (w_hat + n_hat * p.dt)
    # k = 0 (Eq. avg): the mean flow obeys d<v>/dt = (a - 1)<v> + <f_v>; the same scheme
    # gives v^(0) <- exp((a - 1) dt) DFT[v + dt f_v](0)
    g0 = np.exp((p.a - 1.0) * p.dt)
    v0x = g0 * np.real(dft(vx + fvx * p.dt)[0, 0])
    v0y = g0 * np.real(dft(vy + fvy * p.dt)[0, 0])
    w_new, vx_hat, vy_hat = _post_process(w_naive, (v0x, v0y), p)
    # the new velocity in real space, from its (stream-function) spectrum
    return State(np.real(idft(vx_hat)), np.real(idft(vy_hat)), w_new)


def run(s: State, K: np.ndarray, p: Params, nsteps: int, **kw) -> State:
    for _ in range(nsteps):
        s = step(s, K, p, **kw)
    return s


def project_velocity(vx: np.ndarray, vy: np.ndarray, p: Params, dft=dft2, idft=idft2) -> State:
    """Initial state from a real velocity field (reading c6).

    omega^ = i k x v^ = i(kx v^y - ky v^x); then the projection that ends each step with
    v^(0) = DFT[v](0), which zeroes omega^(0), dealiases, Hermitian-averages and rebuilds v
    from the stream function, so the state is divergence-free and band-limited.
    """
    KX, KY, _ = wavenumbers(p)
    Vx, Vy = dft(vx), dft(vy)
    w_hat = 1j * (KX * Vy - KY * Vx)
    w_new, vx_hat, vy_hat = _post_process(w_hat, (np.real(Vx[0, 0]), np.real(Vy[0, 0])), p)
    return State(np.real(idft(vx_hat)), np.real(idft(vy_hat)), w_new)


def from_spectral(w_hat: np.ndarray, v0: tuple, p: Params, idft=idft2) -> State:
    """State whose velocity is the stream-function velocity of w_hat plus mean v^(0) = v0."""
    KX, KY, M2 = wavenumbers(p)
    keep = M2 > 0
    k2 = KX * KX + KY * KY
    psi = np.zeros_like(w_hat)
    psi[keep] = w_hat[keep] / k2[keep]
    vx_hat = 1j * KY * psi
    vy_hat = -1j * KX * psi
    vx_hat[0, 0] = v0[0]
    vy_hat[0, 0] = v0[1]
    return State(np.real(idft(vx_hat)), np.real(idft(vy_hat)), w_hat.copy())


# ----------------------------------------------------------------------------------------
# Diagnostics
# ----------------------------------------------------------------------------------------

def vorticity(s: State, idft=idft2) -> np.ndarray:
    return np.real(idft(s.w_hat))


def vortex_order_parameter(vx, vy, p: Params, center=(0.0, 0.0)) -> float:
    """Psi = (sum|e_theta . v| / sum|v| - 2/pi) / (1 - 2/pi), summed over the whole box
    (Sec. III.C).  e_theta = (-(y - yc), x - xc)/r; at r = 0 it is taken as 0 (reading c12)."""
    n = p.n
    c = (np.arange(n, dtype=np.float64) - n // 2) * p.dx
    X, Y = np.meshgrid(c - center[0], c - center[1], indexing="xy")
    r = np.hypot(X, Y)
    with np.errstate(invalid="ignore", divide="ignore"):
        etx = np.where(r > 0, -Y / r, 0.0)
        ety = np.where(r > 0, X / r, 0.0)
    num = np.sum(np.abs(etx * vx + ety * vy))
    den = np.sum(np.hypot(vx, vy))
    return float((num / den - 2.0 / np.pi) / (1.0 - 2.0 / np.pi))


def shell_spectrum(s: State, p: Params, nbins: int, dft=dft2) -> np.ndarray:
    """E(s) = (2N^2)^-1 sum over modes with round(|m|) = s of |v^(m)|^2 (reading c11)."""
    n = p.n
    MX, MY = index_grid(n)
    shell = np.rint(np.sqrt((MX * MX + MY * MY).astype(np.float64))).astype(np.int64)
    e = np.abs(dft(s.vx)) ** 2 + np.abs(dft(s.vy)) ** 2
    out = np.zeros(nbins)
    sel = shell < nbins
    np.add.at(out, shell[sel], e[sel])
    return out / (2.0 * n * n)


def diagnostics(s: State, p: Params, center=(0.0, 0.0), nbins: int | None = None) -> dict:
    n = p.n
    omega = vorticity(s)
    d = dict(
        energy=float(np.sum(s.vx ** 2 + s.vy ** 2) / (2.0 * n * n)),
        enstrophy=float(np.sum(omega ** 2) / (2.0 * n * n)),
        psi=vortex_order_parameter(s.vx, s.vy, p, center),
        mean_vx=float(np.mean(s.vx)),
        mean_vy=float(np.mean(s.vy)),
    )
    if nbins is not None:
        d["spectrum"] = shell_spectrum(s, p, nbins)
    return d


# ----------------------------------------------------------------------------------------
# Dynamics diagnostics of Sec. III.B and Sec. IV.B
# ----------------------------------------------------------------------------------------

def temporal_psd(fields, times, omegas) -> np.ndarray:
    """S(Omega) = N^-2 sum_x |sum_t omega(x, t) exp(-i Omega t)|^2 (Eq. PSD, Sec. III.B),
    for real vorticity snapshots `fields` taken at `times`."""
    n = fields[0].shape[0]
    out = []
    for Om in omegas:
        A = np.zeros((n, n), dtype=complex)
        for w, t in zip(fields, times):
            A += w * np.exp(-1j * Om * t)
        out.append(np.sum(np.abs(A) ** 2) / (n * n))
    return np.array(out)


def dumbbell_order_parameter(omega, p: Params, centres, radius):
    """Psi_2 = |omega(x*_L) + omega(x*_R)| / (|omega(x*_L)| + |omega(x*_R)|) (Sec. IV.B), where
    x*_{L,R} = argmax |omega| over the grid points within `radius` (= D/2) of each cavity
    centre.  Readings: the disc is closed (distance <= radius); ties go to the first point in
    row-major [y][x] order.  Returns (Psi_2, omega(x*_L), omega(x*_R))."""
    n = p.n
    c = (np.arange(n, dtype=np.float64) - n // 2) * p.dx
    X, Y = np.meshgrid(c, c, indexing="xy")
    peaks = []
    for cx, cy in centres:
        region = (X - cx) ** 2 + (Y - cy) ** 2 <= radius * radius
        flat = np.where(region.reshape(-1), np.abs(omega).reshape(-1), -1.0)
        peaks.append(float(omega.reshape(-1)[int(np.argmax(flat))]))
    a, b = peaks
    return abs(a + b) / (abs(a) + abs(b)), a, b


# ----------------------------------------------------------------------------------------
# Lyapunov exponents (Sec. III.C, "Lyapunov analysis"): independent perturbations evolved
# along with the solution, growth rates from QR decompositions (the standard method the
# paper cites: Shimada & Nagashima 1979, Benettin et al. 1980)
# ----------------------------------------------------------------------------------------

def state_vector(s: State, p: Params) -> np.ndarray:
    """The state as a real vector: (Re, Im) of omega^ on the stored half spectrum (columns
    mx = 0..N/4, entries my = 0..N/4 then -N/4..-1, interleaved re/im), then v^(0)."""
    n, M = p.n, p.n // 4
    ky = np.concatenate([np.arange(0, M + 1), np.arange(-M, 0)])
    half = s.w_hat[np.ix_(ky % n, np.arange(M + 1))].T          # [mx][j]
    v0 = (np.real(dft2(s.vx)[0, 0]), np.real(dft2(s.vy)[0, 0]))
    return np.concatenate([np.stack([half.real, half.imag], axis=-1).reshape(-1), np.array(v0)])


def vector_state(u: np.ndarray, p: Params) -> State:
    """Inverse of state_vector: the mx < 0 half of omega^ follows from omega^(-m) = conj
    omega^(m); the velocity is the stream-function velocity plus v^(0)."""
    n, M = p.n, p.n // 4
    NK = 2 * M + 1
    half = u[:-2].reshape(M + 1, NK, 2)
    half = half[..., 0] + 1j * half[..., 1]
    ky = np.concatenate([np.arange(0, M + 1), np.arange(-M, 0)])
    w_hat = np.zeros((n, n), dtype=complex)
    for mx in range(M + 1):
        w_hat[ky % n, mx] = half[mx]
        if mx > 0:
            w_hat[(-ky) % n, (-mx) % n] = np.conj(half[mx])
    return from_spectral(w_hat, (u[-2], u[-1]), p)


def state_weights(p: Params) -> np.ndarray:
    """Weights that make sum_i w_i u_i u'_i the real-space inner product sum_x (omega omega')
    plus v^(0).v'^(0) (Parseval): 1 on the mx = 0 column, 2 on mx > 0 columns (they stand for
    +-mx), 1 on the mean flow."""
    M = p.n // 4
    NK = 2 * M + 1
    w = np.ones((M + 1, NK, 2))
    w[1:] = 2.0
    return np.concatenate([w.reshape(-1), np.ones(2)])


def lyapunov(s: State, K: np.ndarray, p: Params, q0: np.ndarray, eps: float, nsteps: int,
             interval: int):
    """Lyapunov exponents of the trajectory starting at s.  q0: (k, D) initial perturbation
    directions (state_vector layout).  Every `interval` steps each perturbation, evolved as
    the finite difference (step^interval(s + eps q) - step^interval(s)) / eps of the scheme
    of Algorithm 1, is re-orthonormalised by a QR decomposition (weighted inner product of
    state_weights, R with a positive diagonal); the exponents are the accumulated log R_ii
    divided by the elapsed time.  Returns (exponents, rates of the last interval, final base
    state, final orthonormal directions)."""
    if nsteps % interval:
        raise ValueError("nsteps must be a multiple of interval")
    sw = np.sqrt(state_weights(p))

    def orthonormal(A):                       # columns of A (D, k) -> Q (D, k), diag(R)
        Qw, R = np.linalg.qr(sw[:, None] * A)
        sg = np.sign(np.diag(R))
        return (Qw * sg) / sw[:, None], np.abs(np.diag(R))

    Q, _ = orthonormal(np.asarray(q0, dtype=np.float64).T)
    logs = np.zeros(Q.shape[1])
    last = np.zeros(Q.shape[1])
    for _ in range(nsteps // interval):
        u0 = state_vector(s, p)
        perts = [vector_state(u0 + eps * Q[:, i], p) for i in range(Q.shape[1])]
        s = run(s, K, p, interval)
        u1 = state_vector(s, p)
        D = np.stack([(state_vector(run(pi, K, p, interval), p) - u1) / eps for pi in perts], axis=1)
        Q, r = orthonormal(D)
        logs += np.log(r)
        last = np.log(r) / (interval * p.dt)
    return logs / (nsteps * p.dt), last, s, Q.T
