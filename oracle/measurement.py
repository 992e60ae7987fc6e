"""FP64 measurement operator Phi = G F Z and its real adjoint (oracle; test infrastructure).

Follows Sec. 2 of arXiv:1610.08895 (discrete model y = Phi x + n and the
factorisation Phi = G F Z) and Sec. 3 (data split, eq. data-split). Readings of
what the paper leaves open (stated once here, used everywhere):

* Oversampling "k" is the total factor on the grid size: k = 4 means the grid
  is (2 ny) x (2 nx) (Sec. 5 "oversampling ratio k=4").
* Pixel (iy, ix) sits at centred coordinates (iy - ny/2, ix - nx/2). Z places
  x[iy, ix] * c_y[iy] * c_x[ix] at grid cell ((iy - ny/2) mod Ky, (ix - nx/2) mod Kx).
* F is the unnormalised forward DFT exp(-2 pi i k m / K), matching the sign of the
  continuous model (Sec. 2, eq. measurement-eq).
* A point (u, v) in radians per pixel, in [-pi, pi)^2, sits at continuous grid
  coordinate g = (u Kx / 2pi, v Ky / 2pi); u runs along x (columns), v along y (rows).
* G interpolates with a separable Kaiser-Bessel kernel of width J cells (the
  paper cites an 8x8 compact kernel): phi(t) = I0(beta sqrt(1 - (2t/J)^2)) for
  |t| <= J/2, else 0. The taps of a point at g are the cells floor(g) - J/2 + 1
  ... floor(g) + J/2, wrapped modulo K. The weights are not normalised.
* The pre-compensation in Z is c[i] = 1 / phi_hat((i - n/2) / K), with phi_hat the
  continuous Fourier transform of phi (cycles per cell).

With these, Phi x approximates the direct non-uniform DFT
y_m = sum_p x_p exp(-i (u_m (ix - nx/2) + v_m (iy - ny/2))).
"""
import numpy as np
from scipy.special import i0


def kb_beta_default(J, osf=2.0):
    """Default Kaiser-Bessel shape for width J at oversampling ``osf`` per axis.

    Beatty, Nishimura & Pauly (2005), rule for a kernel of width J at grid
    oversampling alpha: beta = pi sqrt((J/alpha)^2 (alpha - 1/2)^2 - 0.8).
    """
    return np.pi * np.sqrt((J / osf) ** 2 * (osf - 0.5) ** 2 - 0.8)


def kb_kernel(t, J, beta):
    """Kaiser-Bessel interpolation weight phi(t), t in grid cells (entries of G)."""
    t = np.asarray(t, dtype=np.float64)
    arg = 1.0 - (2.0 * t / J) ** 2
    out = np.zeros_like(t)
    inside = arg >= 0.0
    out[inside] = i0(beta * np.sqrt(arg[inside]))
    return out


def kb_fourier(xi, J, beta):
    """Continuous Fourier transform of ``kb_kernel``: integral phi(t) exp(-2 pi i xi t) dt.

    Closed form J sinh(z)/z with z = sqrt(beta^2 - (pi J xi)^2) (and sin for
    imaginary z). Used for the pre-compensation in Z (Sec. 2).
    """
    xi = np.asarray(xi, dtype=np.float64)
    z2 = beta ** 2 - (np.pi * J * xi) ** 2
    out = np.empty_like(xi)
    pos = z2 > 0
    neg = z2 < 0
    zero = ~(pos | neg)
    z = np.sqrt(z2[pos])
    out[pos] = J * np.sinh(z) / z
    zn = np.sqrt(-z2[neg])
    out[neg] = J * np.sin(zn) / zn
    out[zero] = J
    return out


def deapodisation(n, K, J, beta):
    """Per-axis pre-compensation factors c[i] = 1/phi_hat((i - n/2)/K) of Z (Sec. 2)."""
    i = np.arange(n, dtype=np.float64)
    return 1.0 / kb_fourier((i - n / 2) / K, J, beta)


class Geometry:
    """Image/grid sizes and interpolation parameters shared by G, F and Z."""

    def __init__(self, ny, nx, J, beta=None, osf=2):
        if osf != 2:
            raise ValueError("the oracle follows the k = 4 (2 per axis) oversampling")
        self.ny, self.nx = int(ny), int(nx)
        self.Ky, self.Kx = 2 * self.ny, 2 * self.nx
        self.J = int(J)
        self.beta = kb_beta_default(J, 2.0) if (beta is None or beta == 0) else float(beta)
        self.cy = deapodisation(self.ny, self.Ky, self.J, self.beta)
        self.cx = deapodisation(self.nx, self.Kx, self.J, self.beta)

    # --- Z and its adjoint -------------------------------------------------
    def zpad(self, x):
        """Z x: pre-compensate and zero-pad the image into the Ky x Kx grid."""
        g = np.zeros((self.Ky, self.Kx), dtype=np.complex128)
        iy = (np.arange(self.ny) - self.ny // 2) % self.Ky
        ix = (np.arange(self.nx) - self.nx // 2) % self.Kx
        g[np.ix_(iy, ix)] = x * self.cy[:, None] * self.cx[None, :]
        return g

    def zpad_adj(self, g):
        """Z^T g: crop the centred ny x nx region and pre-compensate (complex kept)."""
        iy = (np.arange(self.ny) - self.ny // 2) % self.Ky
        ix = (np.arange(self.nx) - self.nx // 2) % self.Kx
        return g[np.ix_(iy, ix)] * self.cy[:, None] * self.cx[None, :]

    # --- F and its adjoint -------------------------------------------------
    @staticmethod
    def fft(g):
        """F: unnormalised 2-D DFT with exp(-2 pi i k m / K) (library FFT as the step)."""
        return np.fft.fft2(g)

    @staticmethod
    def fft_adj(G):
        """F^H: unnormalised 2-D inverse DFT, exp(+2 pi i k m / K), no 1/K."""
        return np.fft.ifft2(G, norm="forward")

    # --- G and its adjoint -------------------------------------------------
    def grid_coords(self, uv):
        uv = np.asarray(uv, dtype=np.float64)
        gx = uv[:, 0] * self.Kx / (2.0 * np.pi)
        gy = uv[:, 1] * self.Ky / (2.0 * np.pi)
        return gx, gy

    def _taps(self, uv):
        gx, gy = self.grid_coords(uv)
        bx = np.floor(gx).astype(np.int64) - self.J // 2 + 1
        by = np.floor(gy).astype(np.int64) - self.J // 2 + 1
        wx = [kb_kernel(gx - (bx + a), self.J, self.beta) for a in range(self.J)]
        wy = [kb_kernel(gy - (by + b), self.J, self.beta) for b in range(self.J)]
        return bx, by, wx, wy

    def degrid(self, grid, uv):
        """G b: interpolate the grid at the points uv with J x J taps (Sec. 2)."""
        bx, by, wx, wy = self._taps(uv)
        out = np.zeros(len(bx), dtype=np.complex128)
        for b in range(self.J):
            ky = (by + b) % self.Ky
            for a in range(self.J):
                kx = (bx + a) % self.Kx
                out += wy[b] * wx[a] * grid[ky, kx]
        return out

    def grid(self, vis, uv):
        """G^T v: scatter the values v onto the grid with the same J x J weights."""
        bx, by, wx, wy = self._taps(uv)
        vis = np.asarray(vis, dtype=np.complex128)
        size = self.Ky * self.Kx
        re = np.zeros(size)
        im = np.zeros(size)
        for b in range(self.J):
            ky = (by + b) % self.Ky
            for a in range(self.J):
                kx = (bx + a) % self.Kx
                w = wy[b] * wx[a]
                idx = ky * self.Kx + kx
                re += np.bincount(idx, weights=w * vis.real, minlength=size)
                im += np.bincount(idx, weights=w * vis.imag, minlength=size)
        return (re + 1j * im).reshape(self.Ky, self.Kx)

    # --- G with direction-dependent effects (DDEs) ---------------------------
    # Sec. 2: the sparse G "models the compact support DDEs as a convolution in the
    # Fourier domain" on top of the interpolation. Row m of the DDE-aware G is the J x J
    # interpolation kernel of point m convolved with that point's d x d Fourier-domain
    # DDE kernel D_m (d odd, offsets -h .. h with h = (d - 1)/2, [ky offset][kx offset]):
    #   (G b)_m = sum_k D_m[k] sum_c phi_m(c - k) b[c] = sum_k D_m[k] (G (b shifted by -k))_m,
    # written below as that sum of d^2 plain interpolations of the shifted grid.
    def degrid_dde(self, grid, uv, dde):
        """G b with DDE-aware rows: dde is complex [M][d][d] (Sec. 2)."""
        dde = np.asarray(dde, dtype=np.complex128)
        d = dde.shape[1]
        h = (d - 1) // 2
        out = np.zeros(len(uv), dtype=np.complex128)
        for i in range(d):
            for j in range(d):
                shifted = np.roll(grid, (-(i - h), -(j - h)), axis=(0, 1))   # shifted[c] = grid[c + k]
                out += dde[:, i, j] * self.degrid(shifted, uv)
        return out

    def grid_dde(self, vis, uv, dde):
        """G^H v for the DDE-aware G: the adjoint of each term of degrid_dde."""
        dde = np.asarray(dde, dtype=np.complex128)
        vis = np.asarray(vis, dtype=np.complex128)
        d = dde.shape[1]
        h = (d - 1) // 2
        out = np.zeros((self.Ky, self.Kx), dtype=np.complex128)
        for i in range(d):
            for j in range(d):
                out += np.roll(self.grid(np.conj(dde[:, i, j]) * vis, uv), (i - h, j - h), axis=(0, 1))
        return out

    # --- Phi and its real adjoint -----------------------------------------
    def phi(self, x, uv):
        """Phi x = G F Z x for a real image x (Sec. 2)."""
        return self.degrid(self.fft(self.zpad(x)), uv)

    def phi_adj(self, y, uv):
        """Re(Phi^H y) = Re(Z^T F^H G^T y): the adjoint of Phi as a map R^N -> C^M."""
        return np.real(self.zpad_adj(self.fft_adj(self.grid(y, uv))))

    def phi_adj_at(self, y, uv, pixels):
        """Re(Phi^H y) at the listed pixels (iy, ix), one pixel at a time.

        Written out from Phi^H = Z^T F^H G^T for a single output: the entry at pixel
        p is c_y c_x sum_m y_m A_m B_m with A_m = sum_a phi(g_x - k_a) exp(+2 pi i k_a l_x / K_x)
        over the x taps of point m (B_m likewise in y) and l the centred coordinates.
        Linear in the number of points; used where a full grid is too large to form.
        """
        bx, by, wx, wy = self._taps(uv)
        y = np.asarray(y, dtype=np.complex128)
        out = []
        for iy, ix in pixels:
            lx, ly = ix - self.nx // 2, iy - self.ny // 2
            a = sum(wx[k] * np.exp(2j * np.pi * (bx + k) * lx / self.Kx) for k in range(self.J))
            b = sum(wy[k] * np.exp(2j * np.pi * (by + k) * ly / self.Ky) for k in range(self.J))
            out.append(np.real(self.cy[iy] * self.cx[ix] * np.sum(y * a * b)))
        return np.array(out)

