"""Seeded synthetic radar scenes for the distributed-imaging signal model (Eq. 1).

Geometry (Section II): Q sensors on a circle of radius R around a square pixel
grid, each with one transmitter and an M-element uniform linear receive array
(lambda/2 spacing at the carrier, tangential to the circle, centred on the
transmitter).  Each sensor transmits an LFM chirp of bandwidth BW starting at
f_c and hears only its own echo.  After dechirping, fast-time sample k of
receiver m for a point at pixel n with round-trip delay tau is

    exp(j 2 pi tau (f_c + BW k / K)),

so column n of the forward operator A_q (Eq. 1) holds these KM entries, row
index r = m K + k.  The residual-video-phase term is dropped and the chirp
duration cancels.  Pixel n sits at the centre of its cell, row-major in (y, x).

Operators are returned pixel-major (shape (N, KM), complex64): column n of A_q
is the contiguous row ``A[n]``.  Scenes draw per-sensor reflectivity magnitudes
(aspect dependence: every target is seen by each sensor with probability p) and
circular complex Gaussian noise at a given SNR.  This module draws inputs only;
it holds none of the solver's arithmetic.
"""
from dataclasses import dataclass, field
import numpy as np

from .rng import Stream

C0 = 299_792_458.0

# stream ids: one per kind of random draw, so that changing one count never
# shifts another draw
_S_PIX, _S_AMP, _S_VIS, _S_NOISE, _S_CLUSTER, _S_SIZE = 1, 2, 3, 4, 5, 6


@dataclass(frozen=True)
class Geometry:
    Q: int            # sensors
    M: int            # receive antennas per sensor
    K: int            # fast-time samples per chirp
    nx: int           # pixels per side (N = nx * nx)
    cell: float       # pixel pitch [m]
    radius: float     # sensor circle radius [m]
    fc: float         # chirp start frequency [Hz]
    bw: float         # chirp bandwidth [Hz]
    ny: int = None    # rows of pixels (default nx); only unstructured problems set it

    @property
    def N(self):
        return self.nx * (self.nx if self.ny is None else self.ny)

    @property
    def KM(self):
        return self.K * self.M


def pixel_centres(g: Geometry):
    L = g.nx * g.cell
    c = (np.arange(g.nx) + 0.5) * g.cell - L / 2
    X, Y = np.meshgrid(c, c)            # row-major in (y, x)
    return X.ravel(), Y.ravel()


def sensor_positions(g: Geometry, q: int):
    """Transmitter position and the M receiver positions of sensor q."""
    th = 2.0 * np.pi * q / g.Q
    tx = g.radius * np.array([np.cos(th), np.sin(th)])
    tangent = np.array([-np.sin(th), np.cos(th)])
    d = C0 / (2.0 * g.fc)
    off = (np.arange(g.M) - (g.M - 1) / 2.0) * d
    rx = tx[None, :] + off[:, None] * tangent[None, :]
    return tx, rx


def delays(g: Geometry, q: int):
    """Round-trip delays tau[m, n] (seconds), transmitter -> pixel -> receiver m."""
    px, py = pixel_centres(g)
    tx, rx = sensor_positions(g, q)
    d_tx = np.hypot(px - tx[0], py - tx[1])
    d_rx = np.hypot(px[None, :] - rx[:, 0:1], py[None, :] - rx[:, 1:2])
    return (d_tx[None, :] + d_rx) / C0


def operator(g: Geometry, q: int, chunk: int = 2048) -> np.ndarray:
    """A_q pixel-major, complex64, shape (N, KM); phases formed in float64."""
    tau = delays(g, q)                                   # (M, N)
    f = g.fc + g.bw * np.arange(g.K) / g.K               # (K,)
    out = np.empty((g.N, g.KM), dtype=np.complex64)
    for n0 in range(0, g.N, chunk):
        t = tau[:, n0:n0 + chunk].T                      # (n, M)
        cyc = t[:, :, None] * f[None, None, :]           # cycles, (n, M, K)
        cyc -= np.floor(cyc)
        ph = 2.0 * np.pi * cyc
        out[n0:n0 + chunk] = (np.cos(ph) + 1j * np.sin(ph)).reshape(t.shape[0], -1)
    return out


@dataclass
class Scene:
    geom: Geometry
    A: list                 # Q arrays, (N, KM) complex64, pixel-major
    y: list                 # Q arrays, (KM,) complex64
    x_true: np.ndarray      # (Q, N) float64 per-sensor reflectivity magnitudes
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def xG_true(self):
        """Composite ground truth: the sum of the per-sensor images."""
        return self.x_true.sum(axis=0)


def point_targets(g: Geometry, seed: int, n_targets: int, amp=(0.5, 1.0), p_vis=0.8):
    """Per-sensor magnitudes of n_targets point targets at distinct random pixels."""
    pix = Stream(seed, _S_PIX).permutation(g.N)[:n_targets]
    a = Stream(seed, _S_AMP).uniform(n_targets, *amp)
    vis = Stream(seed, _S_VIS).uniform(n_targets * g.Q).reshape(g.Q, n_targets) < p_vis
    x = np.zeros((g.Q, g.N))
    for q in range(g.Q):
        x[q, pix[vis[q]]] = a[vis[q]]
    return x


def cluster_targets(g: Geometry, seed: int, n_clusters: int, amp=(0.3, 1.0), p_vis=0.7,
                    max_size=9):
    """Clusters of 1..max_size pixels inside a 3x3 neighbourhood; one magnitude
    per cluster; each cluster visible to each sensor with probability p_vis."""
    centre = Stream(seed, _S_PIX).permutation(g.N)[:n_clusters]
    size = 1 + Stream(seed, _S_SIZE).integers(n_clusters, max_size)
    a = Stream(seed, _S_AMP).uniform(n_clusters, *amp)
    vis = Stream(seed, _S_VIS).uniform(n_clusters * g.Q).reshape(g.Q, n_clusters) < p_vis
    nb = Stream(seed, _S_CLUSTER)
    offs = np.array([(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
    x = np.zeros((g.Q, g.N))
    for c in range(n_clusters):
        cy, cx = divmod(int(centre[c]), g.nx)
        order = nb.permutation(9)
        # the centre pixel first, then random neighbours
        order = np.concatenate([[4], order[order != 4]])[: size[c]]
        for o in order:
            yy, xx = cy + offs[o][0], cx + offs[o][1]
            if 0 <= yy < g.nx and 0 <= xx < g.nx:
                n = yy * g.nx + xx
                for q in range(g.Q):
                    if vis[q, c]:
                        x[q, n] = a[c]
    return x


def measure(A, x_true, snr_db, seed):
    """y_q = A_q x_q + w_q (Eq. 1); w_q circular Gaussian with
    sigma^2 = ||A_q x_q||^2 / KM * 10^(-SNR/10).  Products in float64."""
    return add_noise([Aq.astype(np.complex128).T @ x_true[q] for q, Aq in enumerate(A)], snr_db, seed)


def add_noise(cleans, snr_db, seed):
    """The noise of measure() added to given noiseless products A_q x_q
    (complex128, one per sensor), for operators too large to hold on the host."""
    ns = Stream(seed, _S_NOISE)
    ys = []
    for clean in cleans:
        clean = np.asarray(clean, dtype=np.complex128)
        KM = clean.shape[0]
        wr, wi = ns.normal(KM), ns.normal(KM)   # drawn even when silent: fixed stream use
        if snr_db is None:
            y = clean
        else:
            sig2 = float(np.vdot(clean, clean).real) / KM * 10.0 ** (-snr_db / 10.0)
            y = clean + np.sqrt(sig2 / 2.0) * (wr + 1j * wi)
        ys.append(y.astype(np.complex64))
    return ys


def lambda_max(A, y, mu=1.0):
    """max_q || mu Re(A_q^H y_q) ||_inf in float64: the smallest lambda for which
    x = 0 satisfies a single sensor's optimality; the scale of the lambda rule."""
    return max(float(np.max(np.abs(mu * (Aq.astype(np.complex128).conj()
                                          @ yq.astype(np.complex128)).real)))
               for Aq, yq in zip(A, y))
