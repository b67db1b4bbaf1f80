"""Small numpy lattice toolkit used only by the tests.

Written independently of both the oracle and the CUDA path, to restate
definitions a second way (finite-difference gradients, the diagonal-subgroup
form of the iteration, brute-force checks).  Lattice-shaped arrays use axes
(t, z, y, x) so that the flat lexicographic site index s = x + Lx*(y + Ly*(z + Lz*t))
is a plain reshape.
"""

import numpy as np

# direction d = 0..3 (x, y, z, t) -> numpy lattice axis
AX = {0: 3, 1: 2, 2: 1, 3: 0}


def lat_shape(dims):
    Lx, Ly, Lz, Lt = dims
    return (Lt, Lz, Ly, Lx)


def to_lat(links, dims):
    """complex [4][V][3][3] -> [4][Lt][Lz][Ly][Lx][3][3]."""
    return np.asarray(links).reshape((4,) + lat_shape(dims) + (3, 3))


def from_lat(U):
    return U.reshape(4, -1, 3, 3)


def shift(a, d, n):
    """Field value at x + n*d_hat (periodic) for an array with lattice axes first."""
    return np.roll(a, -n, axis=AX[d])


def dag(a):
    return np.conj(np.swapaxes(a, -1, -2))


def mm(*ms):
    r = ms[0]
    for m in ms[1:]:
        r = np.einsum("...ij,...jk->...ik", r, m)
    return r


def tr(a):
    return np.einsum("...ii->...", a)


def plaquette(U, mu, nu):
    """P_munu(x) = U_mu(x) U_nu(x+mu) U_mu^dag(x+nu) U_nu^dag(x) for all x."""
    return mm(U[mu], shift(U[nu], mu, 1), dag(shift(U[mu], nu, 1)), dag(U[nu]))


def rectangle(U, mu, nu):
    """2x1 loop: two steps along mu, one along nu, back two along mu, back one along nu."""
    return mm(U[mu], shift(U[mu], mu, 1), shift(U[nu], mu, 2),
              dag(shift(shift(U[mu], mu, 1), nu, 1)), dag(shift(U[mu], nu, 1)), dag(U[nu]))


def gell_mann_generators():
    """T^a = -(i/2) lambda^a: traceless anti-Hermitian, Tr(T^a T^b) = -delta/2."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j; l[1][1, 0] = 1j
    l[2][0, 0] = 1; l[2][1, 1] = -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j; l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j; l[6][2, 1] = 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3); l[7][2, 2] = -2 / np.sqrt(3)
    return -0.5j * l


def expm_eigh(X):
    """exp of an anti-Hermitian X via the eigendecomposition of H = -iX."""
    H = -1j * X
    H = 0.5 * (H + dag(H))
    w, v = np.linalg.eigh(H)
    return mm(v, np.exp(1j * w)[..., :, None] * dag(v))


def colour_mask(dims, mu, c):
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                             indexing="ij")
    xs = {0: x, 1: y, 2: z, 3: t}
    col = 2 * xs[mu]
    for nu in range(4):
        if nu != mu:
            col = col + xs[nu]
    return (col % 4) == c


def label_nearest_centre(trace):
    """Z(3) label as the centre element nearest to Tr U: argmax_n Re(e^{-2 pi i n/3} Tr U)."""
    ns = np.array([0, 1, -1])
    scores = np.stack([np.real(np.exp(-2j * np.pi * n / 3) * trace) for n in ns], axis=-1)
    return ns[np.argmax(scores, axis=-1)]
