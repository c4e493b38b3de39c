"""Seeded synthetic inputs for the MSFV solve (no method arithmetic here).

This module only draws random numbers and lays out problem descriptions. It is
shared by the tests, the benchmark and the oracle checks so that both sides of
a parity comparison see identical inputs; it holds none of the arithmetic of
the multiscale method itself.

Workloads (the DC-resistivity survey of Sec. 2.1 / Sec. 5, with synthetic
conductivities standing in for the paper's block and SEG/EAGE models):

* ``m``: log-conductivity on cells, a Gaussian random field (squared-exponential
  covariance of a given correlation length, mean 0, std 1) drawn by periodic
  spectral synthesis on a grid padded 2x per axis, cropped and standardised;
  optional box anomalies of +/- a given amplitude are added on top.
* sources: dipoles, +amp at one cell and -amp at another (Sec. 2.1, Eq. DCR,
  point electrodes); in 3D they sit on the top layer (surface electrodes).
* receivers: point receivers that sample the cell value; in 3D on the top
  layer (surface measurements, Sec. 2.1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Sequence

import numpy as np


@dataclass
class Problem:
    """Mesh, coarsening, sources and receivers of one MSFV instance.

    Cell index convention: ``idx = i0 + n0*(i1 + n1*i2)`` (axis 0 fastest), the
    unit square / cube, ``h[a] = 1/n[a]``.
    """

    n: tuple                 # cells per axis, len 2 or 3
    coarsen: int             # coarsening factor c (must divide every n[a])
    src_pos: np.ndarray      # (Ns,) int64 cell receiving +amp
    src_neg: np.ndarray      # (Ns,) int64 cell receiving -amp
    src_amp: np.ndarray      # (Ns,) float64
    rec_cell: np.ndarray     # (Nr,) int64 cells sampled by the receivers
    name: str = ""
    source_bases: bool = False   # add one source basis function per source (Sec. 3.2)
    nodal: bool = False          # nodal Galerkin variant: sources / receivers index the
                                 # (n+1)^d nodes, m the n^d cells
    oversample: int = 0          # oversampling width w of the dual edge / face problems
                                 # (cells on each side, normal to the entity; 0: none)

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def N(self) -> int:
        return int(np.prod(self.n))

    @property
    def n_src(self) -> int:
        return int(len(self.src_pos))

    @property
    def n_rec(self) -> int:
        return int(len(self.rec_cell))

    @property
    def h(self) -> tuple:
        return tuple(1.0 / v for v in self.n)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian_random_field(n: Sequence[int], corr_len: float, seed: int) -> np.ndarray:
    """Standardised GRF on the cell centres of the unit box, flattened (axis 0 fastest).

    Periodic spectral synthesis on a 2x padded grid: white complex noise times the
    square root of the squared-exponential spectral density exp(-(k*l)^2/2),
    inverse FFT, crop to the unit box, rescale to mean 0 / std 1.
    """
    rng = _rng(seed)
    n = tuple(int(v) for v in n)
    pad = tuple(2 * v for v in n)
    # numpy arrays are indexed [i_{d-1}, ..., i_0] so that C order = axis 0 fastest
    shape = pad[::-1]
    noise = rng.standard_normal(shape)
    spec = np.fft.fftn(noise)
    k2 = np.zeros(shape)
    for ax_np, npad in enumerate(shape):
        a = len(shape) - 1 - ax_np             # mesh axis of this numpy axis
        hh = 1.0 / n[a]
        kk = 2.0 * np.pi * np.fft.fftfreq(npad, d=hh)
        sh = [1] * len(shape)
        sh[ax_np] = npad
        k2 = k2 + (kk.reshape(sh)) ** 2
    filt = np.exp(-0.25 * k2 * corr_len ** 2)   # sqrt of exp(-k^2 l^2 / 2)
    field_ = np.real(np.fft.ifftn(spec * filt))
    crop = field_[tuple(slice(0, v) for v in shape[::-1][::-1])] if False else field_[
        tuple(slice(0, v) for v in n[::-1])]
    crop = crop - crop.mean()
    sd = crop.std()
    if sd > 0:
        crop = crop / sd
    return np.ascontiguousarray(crop).reshape(-1).astype(np.float64)


def add_box(m: np.ndarray, n: Sequence[int], centre: Sequence[float], side: float,
            amp: float) -> np.ndarray:
    """Add ``amp`` to every cell whose centre lies in the axis-aligned box."""
    n = tuple(int(v) for v in n)
    out = m.copy().reshape(n[::-1])
    grids = np.meshgrid(*[(np.arange(v) + 0.5) / v for v in n[::-1]], indexing="ij")
    mask = np.ones(out.shape, dtype=bool)
    for ax_np, g in enumerate(grids):
        a = len(n) - 1 - ax_np
        mask &= np.abs(g - centre[a]) <= 0.5 * side
    out[mask] += amp
    return out.reshape(-1)


def cell_index(n: Sequence[int], coords: np.ndarray) -> np.ndarray:
    """Flat index of integer cell coordinates ``coords[..., a]`` (axis 0 fastest)."""
    idx = np.zeros(coords.shape[:-1], dtype=np.int64)
    stride = 1
    for a, v in enumerate(n):
        idx += coords[..., a].astype(np.int64) * stride
        stride *= int(v)
    return idx


def _distinct_cells(rng, n, count, top_layer: bool) -> np.ndarray:
    n = tuple(int(v) for v in n)
    if top_layer:
        plane = int(np.prod(n[:-1]))
        if count > plane:
            raise ValueError("not enough top-layer cells")
        pick = rng.choice(plane, size=count, replace=False).astype(np.int64)
        return pick + plane * (n[-1] - 1)
    N = int(np.prod(n))
    return rng.choice(N, size=count, replace=False).astype(np.int64)


def make_problem(n: Sequence[int], coarsen: int, n_src: int, n_rec: int, seed: int,
                 top_layer: bool | None = None, name: str = "",
                 source_bases: bool = False, nodal: bool = False,
                 oversample: int = 0) -> Problem:
    """Dipole sources and point receivers at seeded random distinct cells (nodes of the
    (n+1)^d node lattice when nodal)."""
    n = tuple(int(v) for v in n)
    rng = _rng(seed + 7919)
    if top_layer is None:
        top_layer = len(n) == 3
    lat = tuple(v + 1 for v in n) if nodal else n
    ends = _distinct_cells(rng, lat, 2 * n_src, top_layer)
    src_pos = ends[:n_src].copy()
    src_neg = ends[n_src:].copy()
    rec = np.sort(_distinct_cells(rng, lat, n_rec, top_layer))
    return Problem(n=n, coarsen=int(coarsen), src_pos=src_pos, src_neg=src_neg,
                   src_amp=np.ones(n_src), rec_cell=rec, name=name,
                   source_bases=bool(source_bases), nodal=bool(nodal),
                   oversample=int(oversample))


# ---------------------------------------------------------------------------
# Named workloads (shapes and distributions of the configurations studied)
# ---------------------------------------------------------------------------

def config_2d_64(seed: int = 1):
    """2D, 64x64 cells, c=8, GRF l=0.1, one dipole, 32 receivers."""
    prob = make_problem((64, 64), 8, 1, 32, seed, top_layer=False, name="2d_64x64_c8_s1_r32")
    m = gaussian_random_field(prob.n, 0.1, seed)
    return prob, m


def config_3d_128(seed: int = 2, n: int = 128, coarsen: int = 8):
    """3D, n^3 cells (128 by default), c=8 (by default), GRF l=0.15 plus two +/-2 boxes,
    16 dipoles and 512 receivers on the top layer."""
    nn = (n, n, n)
    prob = make_problem(nn, coarsen, 16, 512 if n >= 32 else min(512, n * n // 2), seed,
                        top_layer=True, name=f"3d_{n}^3_c{coarsen}_s16_r512")
    m = gaussian_random_field(nn, 0.15, seed)
    m = add_box(m, nn, (0.3, 0.5, 0.6), 0.2, +2.0)
    m = add_box(m, nn, (0.7, 0.5, 0.6), 0.2, -2.0)
    return prob, m


def noise_like(shape, scale: float, seed: int) -> np.ndarray:
    """Seeded Gaussian noise (used for 1% data noise and random directions)."""
    return scale * _rng(seed).standard_normal(shape)


def gaussian_random_field_device(n: Sequence[int], corr_len: float, seed: int, device):
    """The same recipe as ``gaussian_random_field`` (2x padded periodic spectral synthesis,
    squared-exponential spectrum, crop, standardise) drawn with torch on a device, for
    meshes whose host-side FFT would dominate a benchmark's set-up (up to 256^3).  Its
    random numbers differ from the host generator's; it feeds only GPU runs."""
    import torch
    n = tuple(int(v) for v in n)
    shape = tuple(2 * v for v in n[::-1])
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    spec = torch.fft.fftn(torch.randn(shape, generator=g, device=device, dtype=torch.float64))
    k2 = torch.zeros(shape, dtype=torch.float64, device=device)
    for ax_np, npad in enumerate(shape):
        a = len(shape) - 1 - ax_np
        kk = 2.0 * np.pi * torch.fft.fftfreq(npad, d=1.0 / n[a], dtype=torch.float64,
                                            device=device)
        sh = [1] * len(shape)
        sh[ax_np] = npad
        k2 = k2 + kk.reshape(sh) ** 2
    field_ = torch.fft.ifftn(spec * torch.exp(-0.25 * k2 * corr_len ** 2)).real
    crop = field_[tuple(slice(0, v) for v in n[::-1])]
    crop = crop - crop.mean()
    sd = crop.std(unbiased=False)
    if float(sd) > 0:
        crop = crop / sd
    return crop.contiguous().reshape(-1)


@dataclass
class InstanceSpec:
    """One independent instance of a batched or served workload (drawn, not built)."""
    n: tuple
    coarsen: int
    corr_len: float
    n_src: int
    n_rec: int
    seed: int

    def problem(self) -> Problem:
        return make_problem(self.n, self.coarsen, self.n_src, self.n_rec, self.seed,
                            top_layer=True,
                            name=f"3d_{self.n[0]}^3_c{self.coarsen}_s{self.n_src}")


def batch_instances(count: int = 64, seed: int = 3,
                    sizes=(64, 96, 128, 192), coarsenings=(4, 8, 16)) -> list:
    """Independent 3D instances of uneven dual-cell sizes: fine size drawn uniformly from
    ``sizes`` (per axis, cubic), coarsening from ``coarsenings``, correlation length from
    U[0.05, 0.2], 8-32 dipoles, 256 top-layer receivers."""
    rng = _rng(seed)
    out = []
    for k in range(count):
        n = int(rng.choice(sizes))
        c = int(rng.choice(coarsenings))
        out.append(InstanceSpec(n=(n, n, n), coarsen=c, corr_len=float(rng.uniform(0.05, 0.2)),
                                n_src=int(rng.integers(8, 33)), n_rec=256,
                                seed=int(seed * 100003 + k)))
    return out


@dataclass
class RequestSpec:
    """One served forward + gradient request: arrival time (s), the client session it
    belongs to (requests of one client are successive Gauss-Newton iterations on one
    mesh and survey), and the seed of its model perturbation."""
    rid: int
    arrival: float
    client: int
    iteration: int
    instance: InstanceSpec


def served_requests(rate: float = 50.0, duration: float = 60.0, seed: int = 5,
                    sizes=(32, 64, 128, 256), coarsenings=(4, 8, 16), max_src: int = 64,
                    p_new_client: float = 0.2) -> list:
    """Poisson arrivals at ``rate`` per second over ``duration`` seconds.  A request opens
    a new client with probability ``p_new_client`` (fine size, coarsening and 1..max_src
    dipoles drawn uniformly, its own seeded lognormal field), else it is the next
    Gauss-Newton iteration of a client drawn uniformly from the open ones."""
    rng = _rng(seed)
    t, rid = 0.0, 0
    clients: list = []
    iters: list = []
    out = []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        if not clients or rng.random() < p_new_client:
            n = int(rng.choice(sizes))
            c = int(rng.choice(coarsenings))
            ns = int(rng.integers(1, max_src + 1))
            nr = min(256, n * n // 2)
            clients.append(InstanceSpec(n=(n, n, n), coarsen=c,
                                        corr_len=float(rng.uniform(0.05, 0.2)), n_src=ns,
                                        n_rec=nr, seed=int(seed * 1000003 + len(clients))))
            iters.append(0)
            k = len(clients) - 1
        else:
            k = int(rng.integers(0, len(clients)))
        out.append(RequestSpec(rid=rid, arrival=t, client=k, iteration=iters[k],
                               instance=clients[k]))
        iters[k] += 1
        rid += 1
    return out


def block_model(n: Sequence[int], background: float = 0.0, amp: float = 2.0):
    """Two conductive blocks (log-conductivity background + amp) in a homogeneous
    half-space, for the Gauss-Newton inversion (Sec. 5.1's two-block setting; the
    block geometry is not given there, so: side 0.25, centres (0.3, 0.5, 0.7) and
    (0.7, 0.5, 0.7) in 3D, (0.3, 0.6) and (0.7, 0.6) in 2D)."""
    n = tuple(int(v) for v in n)
    m = np.full(int(np.prod(n)), float(background))
    if len(n) == 3:
        centres = [(0.3, 0.5, 0.7), (0.7, 0.5, 0.7)]
    else:
        centres = [(0.3, 0.6), (0.7, 0.6)]
    for c in centres:
        m = add_box(m, n, c, 0.25, amp)
    return m
