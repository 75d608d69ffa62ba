"""Seeded synthetic inputs for the Helmholtz Krylov solvers.

This module builds the problems the solvers are run on and nothing else: it
holds none of the solver arithmetic (no SpMV, no inner product, no Krylov
recurrence).  Both the CUDA library and the CPU oracle consume its output.

The paper (Section 1) states the problem as -lap(u) - k^2 u = g on a bounded
domain, k = 2 pi F / c with c varying in space, Dirichlet conditions on part of
the boundary; Section 2 says the matrices come from a finite-element
discretisation stored in CSR.  The paper's own car-cabin matrices (Table 1) are
not public, so this generator produces stand-ins of the same kind: Q1
(trilinear hexahedral) elements on a structured box, at most 27 nonzeros per
row, like the hexahedral Audi3D matrices.

Discretisation (readings of the paper, all stated here):
  * nodes (i, j, k), index i + (nx+1) * (j + (ny+1) * k), position h*(i, j, k);
  * element (ex, ey, ez), index ex + nx * (ey + ny * ez), local node
    a = ax + 2 ay + 4 az at (ex+ax, ey+ay, ez+az);
  * element matrices from the 1-D linear pieces K1 = (1/h)[[1,-1],[-1,1]] and
    M1 = (h/6)[[2,1],[1,2]]:  K_e = K1(x)M1(x)M1 + M1(x)K1(x)M1 + M1(x)M1(x)K1,
    M_e = M1(x)M1(x)M1, top-face B_f = M1(x)M1;
  * per-element speed c_e = 340 (1 + 0.1 U(-1, 1)) m/s;
  * A(w) = K - w^2 M_c + i w B_c with M_c = sum_e M_e / c_e^2 and
    B_c = sum_{top faces} B_f / c_e (Robin impedance condition du/dn = -i k u on
    z = Lz), i.e. A = sum_e (K_e - k_e^2 M_e) + i sum_f k_e B_f;
  * Dirichlet u = 0 on z = 0, eliminated symmetrically: those rows become
    identity rows and their columns are dropped from every other row, so A
    stays exactly symmetric (A == A^T bit for bit);
  * source: lumped Gaussian b_i = h^3 exp(-|x_i - x_s|^2 / (2 sigma^2)),
    sigma = 2h, x_s the box centre, b = 0 on Dirichlet nodes.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

C0 = 340.0  # reference speed of sound, m/s


# ----------------------------------------------------------------------------
# Workload configurations
# ----------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Config:
    """One synthetic workload: a box of nx*ny*nz cubic Q1 elements of size h."""
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    freqs: tuple            # frequencies F in Hz (one for a single solve)
    tol: float = 1e-8       # relative residual target |r|/|b|
    seed: int = 0           # seed of the sound-speed perturbation
    description: str = ""

    @property
    def n(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_elem(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nnz(self) -> int:
        """nnz after Dirichlet elimination on z = 0."""
        nx, ny, nz = self.nx, self.ny, self.nz
        return (3 * nx + 1) * (3 * ny + 1) * (3 * nz - 2) + (nx + 1) * (ny + 1)

    @property
    def F(self) -> float:
        return float(self.freqs[0])


def _ppw_freq(h: float, ppw: float = 10.0) -> float:
    """Frequency giving `ppw` points per wavelength at c = 340 m/s."""
    return C0 / (ppw * h)


CONFIGS = {
    # 20^3 elements on the unit box, F = 1.5 kHz as written (4.5 points per
    # wavelength at h = 0.05; the "~10 points" gloss does not hold there).
    "box20": Config("box20", 20, 20, 20, 0.05, (1500.0,),
                    description="unit box 20x20x20 Q1, F=1500 Hz, c128 BiCGStab to 1e-8"),
    # same box at 10 points per wavelength (680 Hz)
    "box20_10ppw": Config("box20_10ppw", 20, 20, 20, 0.05, (680.0,),
                          description="unit box 20x20x20 Q1, F=680 Hz (10 ppw)"),
    # car-cavity sized 3.0 x 1.5 x 1.25 m, h = 0.025, 10 points per wavelength
    "cavity120": Config("cavity120", 120, 60, 50, 0.025, (_ppw_freq(0.025),),
                        description="3.0x1.5x1.25 m cavity, 120x60x50 Q1, F=1360 Hz"),
    # mixed-precision size 3.0 x 1.5 x 1.2 m, h = 0.015
    "cavity200": Config("cavity200", 200, 100, 80, 0.015, (_ppw_freq(0.015),), tol=1e-10,
                        description="3.0x1.5x1.2 m cavity, 200x100x80 Q1, F=2267 Hz, mixed precision to 1e-10"),
    # frequency sweep: 64 frequencies uniform in [100, 1000] Hz
    "sweep60": Config("sweep60", 60, 30, 25, 0.05,
                      tuple(100.0 + 900.0 * j / 63.0 for j in range(64)),
                      description="3.0x1.5x1.25 m cavity, 60x30x25 Q1, 64 frequencies 100-1000 Hz"),
    # adjoint: 3.0 x 1.5 x 1.2 m, h = 0.0375, 10 points per wavelength
    "adjoint80": Config("adjoint80", 80, 40, 32, 0.0375, (_ppw_freq(0.0375),),
                        description="3.0x1.5x1.2 m cavity, 80x40x32 Q1, F=907 Hz, adjoint gradient"),
}


def tiny_config(nx: int, ny: int, nz: int, h: float = 0.1, F: float = 200.0,
                seed: int = 0, name: str = "tiny") -> Config:
    return Config(name, nx, ny, nz, h, (F,), seed=seed)


# ----------------------------------------------------------------------------
# Element matrices
# ----------------------------------------------------------------------------

def line_matrices(h: float):
    """1-D linear-element stiffness K1 and consistent mass M1."""
    K1 = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    M1 = np.array([[2.0, 1.0], [1.0, 2.0]]) * (h / 6.0)
    return K1, M1


def _local(a: int):
    return a & 1, (a >> 1) & 1, (a >> 2) & 1


def element_matrices(h: float):
    """Q1 hexahedron stiffness K_e (8x8), mass M_e (8x8) and the top-face
    (az = 1) boundary mass B_f (8x8, nonzero only on the 4 top nodes)."""
    K1, M1 = line_matrices(h)
    Ke = np.zeros((8, 8))
    Me = np.zeros((8, 8))
    Bf = np.zeros((8, 8))
    for a in range(8):
        ax, ay, az = _local(a)
        for b in range(8):
            bx, by, bz = _local(b)
            Ke[a, b] = (K1[ax, bx] * M1[ay, by] * M1[az, bz]
                        + M1[ax, bx] * K1[ay, by] * M1[az, bz]
                        + M1[ax, bx] * M1[ay, by] * K1[az, bz])
            Me[a, b] = M1[ax, bx] * M1[ay, by] * M1[az, bz]
            if az == 1 and bz == 1:
                Bf[a, b] = M1[ax, bx] * M1[ay, by]
    return Ke, Me, Bf


# ----------------------------------------------------------------------------
# Assembly on the structured box
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    """Assembled Helmholtz problem on a box (CSR, int32 indices).

    K, Mc, Bc are real float64 value arrays on one shared pattern; the complex
    system matrix at angular frequency w is K - w^2 Mc + i w Bc.
    """
    cfg: Config
    c: np.ndarray            # per-element speed, float64[E]
    rowptr: np.ndarray       # int32[n+1]
    colind: np.ndarray       # int32[nnz]
    K: np.ndarray            # float64[nnz]
    Mc: np.ndarray           # float64[nnz]
    Bc: np.ndarray           # float64[nnz]
    dirichlet: np.ndarray    # bool[n]
    coords: np.ndarray       # float64[n, 3]
    eliminated: bool

    @property
    def n(self) -> int:
        return self.rowptr.size - 1

    @property
    def nnz(self) -> int:
        return self.colind.size


def _stencil_values(cfg: Config, c: np.ndarray, with_dirichlet: bool):
    nx, ny, nz, h = cfg.nx, cfg.ny, cfg.nz, cfg.h
    Ke, Me, Bf = element_matrices(h)
    inv_c2 = 1.0 / (c * c)
    inv_c = 1.0 / c
    n = cfg.n
    kk, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    ii = ii.ravel(); jj = jj.ravel(); kk = kk.ravel()
    # offsets ordered (dk, dj, di) lexicographically -> increasing column index
    offs = [(di, dj, dk) for dk in (-1, 0, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1)]
    Kv = np.zeros((n, 27)); Mv = np.zeros((n, 27)); Bv = np.zeros((n, 27))
    exist = np.zeros((n, 27), dtype=bool)
    for o, (di, dj, dk) in enumerate(offs):
        exist[:, o] = ((ii + di >= 0) & (ii + di <= nx) & (jj + dj >= 0) & (jj + dj <= ny)
                       & (kk + dk >= 0) & (kk + dk <= nz))
        # elements containing both nodes, visited in increasing element index
        # order (ez, ey, ex ascending) so that (p,q) and (q,p) sum identically.
        for cz in (0, 1):
            az = 1 - cz; bz = az + dk
            if bz not in (0, 1):
                continue
            ez = kk - 1 + cz
            for cy in (0, 1):
                ay = 1 - cy; by = ay + dj
                if by not in (0, 1):
                    continue
                ey = jj - 1 + cy
                for cx in (0, 1):
                    ax = 1 - cx; bx = ax + di
                    if bx not in (0, 1):
                        continue
                    ex = ii - 1 + cx
                    ok = ((ex >= 0) & (ex < nx) & (ey >= 0) & (ey < ny) & (ez >= 0) & (ez < nz))
                    e = np.where(ok, ex + nx * (ey + ny * ez), 0)
                    a = ax + 2 * ay + 4 * az
                    b = bx + 2 * by + 4 * bz
                    Kv[:, o] += np.where(ok, Ke[a, b], 0.0)
                    Mv[:, o] += np.where(ok, Me[a, b] * inv_c2[e], 0.0)
                    if az == 1 and bz == 1:
                        top = ok & (ez == nz - 1)
                        Bv[:, o] += np.where(top, Bf[a, b] * inv_c[e], 0.0)
    dir_node = kk == 0
    if with_dirichlet:
        # drop Dirichlet columns from every row; Dirichlet rows -> identity
        colk = kk[:, None] + np.array([d[2] for d in offs])[None, :]
        exist &= ~(colk == 0)
        exist[dir_node, :] = False
        centre = 13  # offset (0,0,0)
        exist[dir_node, centre] = True
        Kv[dir_node, :] = 0.0; Mv[dir_node, :] = 0.0; Bv[dir_node, :] = 0.0
        Kv[dir_node, centre] = 1.0
    cols = (ii[:, None] + np.array([d[0] for d in offs])[None, :]
            + (nx + 1) * ((jj[:, None] + np.array([d[1] for d in offs])[None, :])
                          + (ny + 1) * (kk[:, None] + np.array([d[2] for d in offs])[None, :])))
    counts = exist.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colind = cols[exist].astype(np.int32)
    coords = np.stack([ii * h, jj * h, kk * h], axis=1).astype(np.float64)
    return (rowptr.astype(np.int32), colind, Kv[exist], Mv[exist], Bv[exist],
            dir_node if with_dirichlet else np.zeros(n, dtype=bool), coords)


def sound_speed(cfg: Config, seed: Optional[int] = None) -> np.ndarray:
    """c_e = 340 (1 + 0.1 U(-1,1)) per element, drawn with numpy's PCG64."""
    rng = np.random.default_rng(cfg.seed if seed is None else seed)
    return C0 * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, cfg.n_elem))


def assemble(cfg: Config, c: Optional[np.ndarray] = None, dirichlet: bool = True) -> Problem:
    """Assemble K, M_c, B_c on the CSR pattern of the box."""
    if c is None:
        c = sound_speed(cfg)
    c = np.asarray(c, dtype=np.float64)
    if c.shape != (cfg.n_elem,):
        raise ValueError("c must have one entry per element")
    rowptr, colind, K, Mc, Bc, dnode, coords = _stencil_values(cfg, c, dirichlet)
    return Problem(cfg, c, rowptr, colind, K, Mc, Bc, dnode, coords, dirichlet)


def omega(F: float) -> float:
    return 2.0 * math.pi * F


def helmholtz_values(prob: Problem, F: float) -> np.ndarray:
    """Complex values of A = K - w^2 M_c + i w B_c on the problem's pattern."""
    w = omega(F)
    return (prob.K - (w * w) * prob.Mc) + 1j * (w * prob.Bc)


def source(prob: Problem, sigma_h: float = 2.0) -> np.ndarray:
    """Lumped Gaussian point source at the box centre (complex128[n])."""
    cfg = prob.cfg
    h = cfg.h
    centre = np.array([cfg.nx * h, cfg.ny * h, cfg.nz * h]) / 2.0
    sigma = sigma_h * h
    d2 = ((prob.coords - centre) ** 2).sum(axis=1)
    g = np.exp(-d2 / (2.0 * sigma * sigma))
    b = (h ** 3) * g
    b[prob.dirichlet] = 0.0
    return b.astype(np.complex128)


def receivers(prob: Problem, count: int = 64, seed: int = 1) -> np.ndarray:
    """`count` distinct non-Dirichlet node indices (sorted), seeded."""
    rng = np.random.default_rng(seed)
    free = np.flatnonzero(~prob.dirichlet)
    return np.sort(rng.choice(free, size=count, replace=False)).astype(np.int64)


# ----------------------------------------------------------------------------
# Element bookkeeping for the sound-speed gradient
# ----------------------------------------------------------------------------

def element_nodes(cfg: Config) -> np.ndarray:
    """int32[E, 8] global node of each element's local node a = ax + 2ay + 4az."""
    nx, ny, nz = cfg.nx, cfg.ny, cfg.nz
    ez, ey, ex = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ex = ex.ravel(); ey = ey.ravel(); ez = ez.ravel()
    out = np.empty((ex.size, 8), dtype=np.int32)
    for a in range(8):
        ax, ay, az = _local(a)
        out[:, a] = (ex + ax) + (nx + 1) * ((ey + ay) + (ny + 1) * (ez + az))
    return out


def element_nnz_map(prob: Problem) -> np.ndarray:
    """int32[E, 64]: CSR slot of (node a, node b) of each element, row-major in
    (a, b); -1 where the pair was eliminated (either node on a Dirichlet row,
    whose entries do not depend on c)."""
    en = element_nodes(prob.cfg)
    rows = en[:, :, None].repeat(8, axis=2).reshape(-1)
    cols = en[:, None, :].repeat(8, axis=1).reshape(-1)
    rowptr = prob.rowptr.astype(np.int64)
    out = np.full(rows.size, -1, dtype=np.int64)
    keep = ~(prob.dirichlet[rows] | prob.dirichlet[cols])
    r = rows[keep]; cc = cols[keep]
    # columns within a row are sorted: binary search inside each row
    start = rowptr[r]; end = rowptr[r + 1]
    lo = start.copy(); hi = end.copy()
    colind = prob.colind
    while True:
        active = lo < hi
        if not active.any():
            break
        mid = (lo + hi) // 2
        v = colind[np.minimum(mid, colind.size - 1)]
        less = active & (v < cc)
        lo = np.where(less, mid + 1, lo)
        hi = np.where(active & ~less, mid, hi)
    if np.any(colind[lo] != cc):
        raise RuntimeError("element pair missing from the CSR pattern")
    out[keep] = lo
    return out.reshape(-1, 64).astype(np.int32)


def slot_elements(prob: Problem, elem_map: Optional[np.ndarray] = None, width: int = 8):
    """Inverse of element_nnz_map: for each CSR slot, the (element, pair)
    contributions, sorted by element index, padded with element -1.
    Returns (elem int32[nnz, width], pair uint8[nnz, width]); pair = 8 a + b."""
    if elem_map is None:
        elem_map = element_nnz_map(prob)
    E = elem_map.shape[0]
    e_idx = np.repeat(np.arange(E, dtype=np.int64), 64)
    ab = np.tile(np.arange(64, dtype=np.int64), E)
    slot = elem_map.reshape(-1).astype(np.int64)
    keep = slot >= 0
    e_idx, ab, slot = e_idx[keep], ab[keep], slot[keep]
    order = np.lexsort((e_idx, slot))
    e_idx, ab, slot = e_idx[order], ab[order], slot[order]
    counts = np.bincount(slot, minlength=prob.nnz)
    if counts.max() > width:
        raise ValueError("more contributions per slot than the table width")
    start = np.zeros(prob.nnz + 1, dtype=np.int64)
    np.cumsum(counts, out=start[1:])
    pos = np.arange(slot.size) - start[slot]
    elem = np.full((prob.nnz, width), -1, dtype=np.int32)
    pair = np.zeros((prob.nnz, width), dtype=np.uint8)
    elem[slot, pos] = e_idx
    pair[slot, pos] = ab
    return elem, pair


def top_elements(cfg: Config) -> np.ndarray:
    """uint8[E]: 1 for elements with a face on z = Lz (the impedance face)."""
    e = np.arange(cfg.n_elem)
    return ((e // (cfg.nx * cfg.ny)) == cfg.nz - 1).astype(np.uint8)


# ----------------------------------------------------------------------------
# Seeded vectors and generic CSR for tests and microbenchmarks
# ----------------------------------------------------------------------------

def complex_vector(n: int, seed: int) -> np.ndarray:
    """Uniform complex entries in the unit square [-1,1]^2, seeded."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(-1.0, 1.0, size=(n, 2))
    return (v[:, 0] + 1j * v[:, 1]).astype(np.complex128)


def random_csr(n: int, max_row: int, seed: int, empty_row_frac: float = 0.1,
               ncols: Optional[int] = None):
    """Random CSR (sorted, distinct columns per row) with a ragged length mix,
    including empty rows; complex values uniform in the unit square."""
    rng = np.random.default_rng(seed)
    ncols = n if ncols is None else ncols
    lens = rng.integers(0, max_row + 1, size=n)
    lens[rng.random(n) < empty_row_frac] = 0
    lens = np.minimum(lens, ncols)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rowptr[1:])
    cols = np.empty(int(rowptr[-1]), dtype=np.int32)
    for i in range(n):
        if lens[i]:
            cols[rowptr[i]:rowptr[i + 1]] = np.sort(rng.choice(ncols, size=lens[i], replace=False))
    vals = complex_vector(int(rowptr[-1]), seed + 1)
    return rowptr.astype(np.int32), cols, vals
