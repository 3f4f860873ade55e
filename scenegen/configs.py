"""Named synthetic workloads.

* ``small_point``: Q=4 sensors on a 10 m circle around a 2 m x 2 m scene of
  32x32 pixels, M=4, K=64 (KM=256), f_c=77 GHz, BW=1 GHz, 8 point targets with
  magnitudes U[0.5, 1], visibility p=0.8 per sensor, 20 dB SNR, rho=1,
  lambda = 0.05 * lambda_max, 300 iterations, seed 0.
* ``paper_scale``: Q=8, M=8, K=256 (KM=2048), 128x128 pixels of 5 cm (the
  paper's cell size), same radar and circle as ``small_point``; 40 clusters of
  1..9 pixels, magnitudes U[0.3, 1], p=0.7, 15 dB SNR; relative-change
  tolerance 1e-4, pixel elimination on.
* mixed-geometry batches (``batch_geometries``, ``batch_scenes``): geometries
  drawn by seed from the 48 combinations of Q in {2, 4, 6, 8}, M in {4, 8},
  K in {128, 256}, N in {48^2, 64^2, 96^2} (radar, circle and 5 cm cells as
  ``paper_scale``), 16 scenes per geometry with 5..60 clusters, visibility
  p in [0.5, 0.9] and 10..25 dB SNR.
* ``precision_twin``: the sensors of the 256x256 precision workload (Q=8,
  M=16, K=512, KM=8192) over a 64x64 crop of 5 cm cells, 8 clusters, p=0.7,
  20 dB: the size the FP64 oracle checks that workload's forms at.
* ``resolved_128``: the paper-scale problem size (Q=8 sensors, N=128x128
  pixels) on a geometry where every sensor resolves the grid on its own, so
  that Eq. 2 has a unique, nonzero minimiser: 8 cm cells (a 10.24 m scene)
  seen from an 8 m circle by sensors with M=256 receivers at 60 GHz, BW=4 GHz,
  K=64 (KM=16384: 2KM = 2N, Gram condition ~8.5e4, as resolved_32's); the
  scene law of ``paper_scale`` (40 clusters of 1..9 pixels, magnitudes
  U[0.3, 1], p=0.7, 15 dB SNR).
* ``resolved_tiny``: a well-posed geometry used by the oracle's pins: 8x8
  pixels of 10 cm seen from 0.6 m by sensors with M=16 antennas and BW=4 GHz
  at 60 GHz (K=16, KM=256 > N), so that every sensor resolves the grid on its
  own and the sharing problem has a unique minimiser.
"""
from dataclasses import dataclass
import numpy as np

from .radar import Geometry, Scene, operator, point_targets, cluster_targets, measure, lambda_max


@dataclass(frozen=True)
class Params:
    mu: float = 1.0
    rho: float = 1.0
    lam_frac: float = 0.05   # lambda = lam_frac * lambda_max  (ignored if lam is set)
    lam: float = None
    Kp: int = 5
    eps_p: float = 1e-5
    eps_abs: float = 1e-4
    eps_rel: float = 1e-2
    iters: int = 300
    tol: float = 1e-4


GEOMS = {
    "small_point": Geometry(Q=4, M=4, K=64, nx=32, cell=2.0 / 32, radius=10.0, fc=77e9, bw=1e9),
    "paper_scale": Geometry(Q=8, M=8, K=256, nx=128, cell=0.05, radius=10.0, fc=77e9, bw=1e9),
    "resolved_tiny": Geometry(Q=3, M=16, K=16, nx=8, cell=0.10, radius=0.6, fc=60e9, bw=4e9),
    # 32x32 grid that every sensor resolves on its own (2KM = 2N, condition ~300):
    # Eq. 2 is well posed, so the iterates converge to a nonzero image
    "resolved_32": Geometry(Q=4, M=32, K=32, nx=32, cell=0.08, radius=2.0, fc=60e9, bw=4e9),
    # Q=8, N=128x128 with every sensor resolving the grid (2KM = 2N, Gram
    # condition ~8.5e4): the paper-scale size of a well-posed Eq. 2
    "resolved_128": Geometry(Q=8, M=256, K=64, nx=128, cell=0.08, radius=8.0, fc=60e9, bw=4e9),
    # the precision workload at its full size (Q=8, M=16, K=512: KM=8192,
    # N=256x256 of 5 cm; operators 8 x 4.3 GB): built on the device
    "precision_256": Geometry(Q=8, M=16, K=512, nx=256, cell=0.05, radius=10.0, fc=77e9, bw=1e9),
    # the precision-form sensors (Q=8, M=16, K=512: KM=8192) over a 64x64 crop
    # of 5 cm cells, the oracle-sized twin of the 256x256 precision workload
    "precision_twin": Geometry(Q=8, M=16, K=512, nx=64, cell=0.05, radius=10.0, fc=77e9, bw=1e9),
}


def operators(g: Geometry):
    """The Q sensors' operators, built on host threads (the per-entry phase
    arithmetic releases the interpreter lock)."""
    if g.Q == 1 or g.N * g.KM < (1 << 22):
        return [operator(g, q) for q in range(g.Q)]
    import os
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=min(g.Q, os.cpu_count() or 1)) as pool:
        return list(pool.map(lambda q: operator(g, q), range(g.Q)))


def scene_law(name: str, g: Geometry, seed: int = 0, n_targets=None):
    """(per-sensor reflectivities x (Q, N), SNR in dB) of the named workload."""
    if name in ("paper_scale", "resolved_128"):
        x = cluster_targets(g, seed, n_targets or 40, amp=(0.3, 1.0), p_vis=0.7)
        snr = 15.0
    elif name == "precision_256":
        x = cluster_targets(g, seed, n_targets or 120, amp=(0.3, 1.0), p_vis=0.7)
        snr = 20.0
    elif name == "precision_twin":
        # 120 targets on 256^2 pixels keep their density on the 64^2 crop
        x = cluster_targets(g, seed, n_targets or 8, amp=(0.3, 1.0), p_vis=0.7)
        snr = 20.0
    elif name == "resolved_32":
        x = cluster_targets(g, seed, n_targets or 10, amp=(0.3, 1.0), p_vis=0.7)
        snr = 25.0
    elif name == "resolved_tiny":
        x = point_targets(g, seed, n_targets or 3, amp=(0.5, 1.0), p_vis=0.8)
        snr = 30.0
    else:
        x = point_targets(g, seed, n_targets or 8, amp=(0.5, 1.0), p_vis=0.8)
        snr = 20.0
    return x, snr


def build_scene(name: str, seed: int = 0, geom: Geometry = None, snr_db="default",
                n_targets=None) -> Scene:
    g = geom or GEOMS[name]
    A = operators(g)
    x, snr = scene_law(name, g, seed, n_targets)
    if snr_db != "default":
        snr = snr_db
    y = measure(A, x, snr, seed)
    return Scene(geom=g, A=A, y=y, x_true=x, seed=seed, meta={"name": name, "snr_db": snr})


def resolve_lambda(scene: Scene, p: Params) -> float:
    if p.lam is not None:
        return float(p.lam)
    return p.lam_frac * lambda_max(scene.A, scene.y, p.mu)


def random_problem(Q, KM, N, seed, snr_db=30.0, k_sparse=3):
    """Unstructured i.i.d. complex Gaussian operators (unit-variance entries),
    complex64 pixel-major, with a sparse per-sensor ground truth.  Used where a
    pin needs generic, well-conditioned operators."""
    from .rng import Stream
    s = Stream(seed, 101)
    A = []
    for q in range(Q):
        re = s.normal(N * KM).reshape(N, KM)
        im = s.normal(N * KM).reshape(N, KM)
        A.append(((re + 1j * im) / np.sqrt(2.0)).astype(np.complex64))
    g = Geometry(Q=Q, M=1, K=KM, nx=N, ny=1, cell=1.0, radius=1.0, fc=1.0, bw=1.0)
    x = np.zeros((Q, N))
    pix = Stream(seed, 102).permutation(N)[:k_sparse]
    amp = Stream(seed, 103).uniform(k_sparse * Q, 0.5, 1.0).reshape(Q, k_sparse)
    for q in range(Q):
        x[q, pix] = amp[q]
    y = measure(A, x, snr_db, seed)
    return Scene(geom=g, A=A, y=y, x_true=x, seed=seed, meta={"name": "random"})


BATCH_Q = (2, 4, 6, 8)
BATCH_M = (4, 8)
BATCH_K = (128, 256)
BATCH_NX = (48, 64, 96)


def batch_geometries(seed: int, count: int = 32):
    """`count` distinct geometries drawn by seed (without repetition) from the
    48 combinations of BATCH_Q x BATCH_M x BATCH_K x BATCH_NX."""
    from .rng import Stream
    combos = [(Q, M, K, nx) for Q in BATCH_Q for M in BATCH_M for K in BATCH_K for nx in BATCH_NX]
    if not 1 <= count <= len(combos):
        raise ValueError(f"count must be in 1..{len(combos)}")
    pick = Stream(seed, 301).permutation(len(combos))[:count]
    return [Geometry(Q=combos[i][0], M=combos[i][1], K=combos[i][2], nx=combos[i][3], cell=0.05, radius=10.0,
                     fc=77e9, bw=1e9) for i in pick]


def batch_scenes(g: Geometry, A, seed: int, S: int = 16):
    """S scenes sharing the operators A of geometry g: 5..60 clusters of
    magnitudes U[0.3, 1], visibility p ~ U[0.5, 0.9], SNR ~ U[10, 25] dB, all
    drawn by seed.  Returns (Y, lams): Y (S, Q, KM) complex64 and the per-scene
    lambda = 0.05 lambda_max."""
    from .rng import Stream
    st = Stream(seed, 302)
    n_cl = 5 + st.integers(S, 56)
    p_vis = st.uniform(S, 0.5, 0.9)
    snr = st.uniform(S, 10.0, 25.0)
    Y, lams = [], []
    for s in range(S):
        sub = 1000 * seed + s
        x = cluster_targets(g, sub, int(n_cl[s]), amp=(0.3, 1.0), p_vis=float(p_vis[s]))
        y = measure(A, x, float(snr[s]), sub)
        Y.append(np.stack(y))
        lams.append(0.05 * lambda_max(A, y))
    return np.stack(Y).astype(np.complex64), lams
