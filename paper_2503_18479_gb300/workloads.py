"""Seeded synthetic inputs shaped like the paper's workloads.

This module only generates inputs: loop geometry, field points, capacitances, frequencies,
drive voltages and targets. It holds none of the method's arithmetic (no Biot-Savart sum, no
inductance, no solve, no superposition), so that the CUDA path and the CPU oracle can both
consume its output without sharing code. Two quantities here are physics in the narrow sense
and are inputs of the method, not steps of it:

* the drive voltage of each loop, V_k = -j w B_inc A_k: the EMF of a uniform incident field
  B_inc along z through the loop's (shoelace) area A_k, the excitation chosen for these
  synthetic runs in place of the paper's excitation coil / birdcage (Sec. III-B), and
* the closed-form self inductance mu0 a (ln(8a/r_w) - 2) of a thin circular loop, which the
  single-loop workload feeds in as L (its 64-gon has oblique segment pairs).

Workloads (all seeded with numpy PCG64):
  single_loop  -- one circular 64-gon loop (radius 50 mm, wire radius 1 mm), 101 frequencies
                  in 60-68 MHz, 32x32 grid at z = 20 mm over +-100 mm, 4 loss points on the
                  grid; the paper's 0D cell (Sec. III-B, IV-A).
  line_8x1     -- 8x1 square loops (side 50 mm, pitch 55 mm, 16 segments a side), 201
                  frequencies, 64x64 grid at z = 20 mm over +-250 mm, 8 loss points above the
                  cell centres at 0.8 x the cell size (Sec. III-C); the paper's 1D MTS.
  array_8x8    -- 8x8 of the same cells at 63.6 MHz, 4 planes of 128x128 points at
                  z = 10/20/30/40 mm over +-250 mm, 64 loss points at z = 40 mm, targets
                  N(0,1) x 1e-6 T; the paper's 2D MTS (Sec. IV-C).
  ragged       -- many independent rectangular arrays with 1..128 ports and 1..16 frequencies.
  array_32x32  -- 32x32 cells (1024 ports), 4 planes of 512x512 points over +-900 mm.
  sroute_array -- inputs of the scattering-parameter route shaped like the 8x8 array driven
                  by one excitation loop (n0 = 65 structure ports, one external port): a
                  reciprocal passive S0 per frequency, per-port fields of z-directed
                  magnetic-dipole form at the array's points, the drive port fed through
                  S_C12, and series RC loads (R, C) on the 64 cell ports. These stand in for
                  a full-wave export; the S-parameters of the loads are computed by the route
                  itself (Eq. 2-3), not here.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

MU0 = 4e-7 * np.pi
PF = 1e-12
MHZ = 1e6


@dataclass
class Structure:
    """One independent structure: loops, field points, frequencies and drive."""
    loop_vtx_off: np.ndarray  # int32 [N+1], local vertex offsets (closed polylines)
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    px: np.ndarray
    py: np.ndarray
    pz: np.ndarray
    R: np.ndarray  # [N] ohm
    omega: np.ndarray  # [F] rad/s
    V: np.ndarray  # complex [F, N] volt
    loss_idx: np.ndarray  # int64 [L], local point indices
    L_self: Optional[np.ndarray] = None  # [N] henry or None (partial-inductance sum)
    pcomp: Optional[np.ndarray] = None  # int8 [P] field component per point (0 z, 1 x, 2 y)
    label: str = ""

    @property
    def n_ports(self) -> int:
        return len(self.loop_vtx_off) - 1

    @property
    def n_points(self) -> int:
        return len(self.px)

    @property
    def n_freq(self) -> int:
        return len(self.omega)

    @property
    def n_loss(self) -> int:
        return len(self.loss_idx)


@dataclass
class Workload:
    name: str
    structures: List[Structure]
    C: np.ndarray  # [n_cfg, N_total] farad
    wire_radius: float
    loss_mode: int = 0  # 0: (|Bz| - t)^2, 1: |Bz - t|^2
    target: Optional[np.ndarray] = None  # concatenated [sum F_s L_s] (per cfg: [n_cfg, ...])
    target_per_cfg: bool = False
    target_rule: Optional[tuple] = None  # ("field_at_C", C_value): target = |Bz| at that C
    meta: dict = field(default_factory=dict)

    @property
    def n_cfg(self) -> int:
        return self.C.shape[0]

    @property
    def n_ports(self) -> int:
        return sum(s.n_ports for s in self.structures)

    @property
    def n_points(self) -> int:
        return sum(s.n_points for s in self.structures)

    @property
    def n_freq(self) -> int:
        return sum(s.n_freq for s in self.structures)

    @property
    def n_loss(self) -> int:
        return sum(s.n_loss for s in self.structures)

    def port_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum([s.n_ports for s in self.structures])]).astype(np.int32)

    def point_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum([s.n_points for s in self.structures])]).astype(np.int64)

    def freq_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum([s.n_freq for s in self.structures])]).astype(np.int32)

    def loss_off(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum([s.n_loss for s in self.structures])]).astype(np.int32)

    def target_off(self) -> np.ndarray:
        """Offsets of each structure's [F_s, L_s] target block in the concatenated array."""
        return np.concatenate([[0], np.cumsum([s.n_freq * s.n_loss for s in self.structures])]).astype(np.int64)

    def structure_target(self, s: int) -> np.ndarray:
        """Target block of structure s: [F, L] (or [n_cfg, F, L] when per configuration)."""
        st = self.structures[s]
        off = self.target_off()
        w = 2 if self.loss_mode == 1 else 1
        if self.target_per_cfg:
            t = self.target.reshape(self.n_cfg, -1)[:, off[s] * w:off[s + 1] * w]
            return t.reshape(self.n_cfg, st.n_freq, st.n_loss, w).squeeze(-1) if w == 1 else \
                t.reshape(self.n_cfg, st.n_freq, st.n_loss, 2)
        t = self.target[off[s] * w:off[s + 1] * w]
        return t.reshape(st.n_freq, st.n_loss) if w == 1 else t.reshape(st.n_freq, st.n_loss, 2)

    def structure_C(self, s: int) -> np.ndarray:
        po = self.port_off()
        return self.C[:, po[s]:po[s + 1]]

    def flat(self) -> dict:
        """Concatenated arrays in the layout of the C ABI (global indices)."""
        ss = self.structures
        vtx_base = np.concatenate([[0], np.cumsum([len(s.vx) for s in ss])])
        pt_base = self.point_off()
        loop_off = [np.zeros(1, np.int32)]
        for i, s in enumerate(ss):
            loop_off.append((s.loop_vtx_off[1:] + vtx_base[i]).astype(np.int32))
        has_L = any(s.L_self is not None for s in ss)
        if has_L and not all(s.L_self is not None for s in ss):
            raise ValueError("L_self must be given for every structure or none")
        has_comp = any(s.pcomp is not None for s in ss)
        return dict(
            port_off=self.port_off(), point_off=self.point_off(), freq_off=self.freq_off(),
            loss_off=self.loss_off(),
            loop_vtx_off=np.concatenate(loop_off).astype(np.int32),
            vx=np.concatenate([s.vx for s in ss]), vy=np.concatenate([s.vy for s in ss]),
            vz=np.concatenate([s.vz for s in ss]),
            px=np.concatenate([s.px for s in ss]), py=np.concatenate([s.py for s in ss]),
            pz=np.concatenate([s.pz for s in ss]),
            loss_idx=np.concatenate([s.loss_idx + pt_base[i] for i, s in enumerate(ss)]).astype(np.int64),
            R=np.concatenate([s.R for s in ss]),
            L_self=np.concatenate([s.L_self for s in ss]) if has_L else None,
            pcomp=np.concatenate([s.pcomp if s.pcomp is not None else np.zeros(s.n_points, np.int8)
                                  for s in ss]).astype(np.int8) if has_comp else None,
            omega=np.concatenate([s.omega for s in ss]),
            V=np.concatenate([s.V.reshape(-1) for s in ss]).astype(np.complex128),
        )


# ---------------------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------------------
def circular_loop(a: float, n_seg: int, cx: float = 0.0, cy: float = 0.0, z: float = 0.0):
    """Regular n_seg-gon inscribed in radius a, counter-clockwise seen from +z."""
    t = 2.0 * np.pi * np.arange(n_seg) / n_seg
    return cx + a * np.cos(t), cy + a * np.sin(t), np.full(n_seg, z)


def square_loop(side: float, seg_per_side: int, cx: float = 0.0, cy: float = 0.0, z: float = 0.0):
    """Square loop, counter-clockwise from the (-h,-h) corner, each side split evenly.

    Vertices of one side share one coordinate exactly, so segment directions are exactly
    axis-aligned (parallel/perpendicular tests are exact)."""
    h = side / 2.0
    step = side / seg_per_side
    i = np.arange(seg_per_side)
    xs = np.concatenate([cx - h + i * step, np.full(seg_per_side, cx + h),
                         cx + h - i * step, np.full(seg_per_side, cx - h)])
    ys = np.concatenate([np.full(seg_per_side, cy - h), cy - h + i * step,
                         np.full(seg_per_side, cy + h), cy + h - i * step])
    return xs, ys, np.full(4 * seg_per_side, z)


def polygon_area(x: np.ndarray, y: np.ndarray) -> float:
    """Signed (shoelace) area of a closed polygon; positive when counter-clockwise."""
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def loops_to_arrays(loops):
    off = np.zeros(len(loops) + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(l[0]) for l in loops])
    vx = np.concatenate([l[0] for l in loops])
    vy = np.concatenate([l[1] for l in loops])
    vz = np.concatenate([l[2] for l in loops])
    return off, vx, vy, vz


def square_array(nx: int, ny: int, side=0.050, pitch=0.055, seg_per_side=16):
    """Cells at ((i - (nx-1)/2) pitch, (j - (ny-1)/2) pitch, 0); port k = j*nx + i."""
    loops = []
    for j in range(ny):
        for i in range(nx):
            loops.append(square_loop(side, seg_per_side, (i - (nx - 1) / 2.0) * pitch,
                                     (j - (ny - 1) / 2.0) * pitch))
    return loops


def grid_plane(n: int, half_span: float, z: float, nx: Optional[int] = None, half_span_y=None,
               cx: float = 0.0, cy: float = 0.0):
    """n x n (or nx x n) linspace grid; point index = iy * nx + ix."""
    nx = nx or n
    hy = half_span if half_span_y is None else half_span_y
    xs = cx + np.linspace(-half_span, half_span, nx)
    ys = cy + np.linspace(-hy, hy, n)
    X, Y = np.meshgrid(xs, ys)
    return X.ravel(), Y.ravel(), np.full(X.size, z)


def drive_uniform_field(loops, omega: np.ndarray, B_inc: float = 1e-6) -> np.ndarray:
    """V[f, k] = -j w_f B_inc A_k (EMF of a uniform field along z, e^{+jwt})."""
    areas = np.array([polygon_area(l[0], l[1]) for l in loops])
    return (-1j * omega[:, None] * B_inc * areas[None, :]).astype(np.complex128)


def circular_loop_inductance(a: float, wire_radius: float) -> float:
    """Thin circular loop without internal inductance: mu0 a (ln(8a/r_w) - 2)."""
    return MU0 * a * (np.log(8.0 * a / wire_radius) - 2.0)


def _structure_from(loops, points, omega, R, loss_idx, L_self=None, label=""):
    off, vx, vy, vz = loops_to_arrays(loops)
    px, py, pz = points
    n = len(loops)
    return Structure(loop_vtx_off=off, vx=vx, vy=vy, vz=vz, px=np.ascontiguousarray(px),
                     py=np.ascontiguousarray(py), pz=np.ascontiguousarray(pz),
                     R=np.full(n, R) if np.isscalar(R) else np.asarray(R, float),
                     omega=np.asarray(omega, float), V=drive_uniform_field(loops, np.asarray(omega, float)),
                     loss_idx=np.asarray(loss_idx, np.int64), L_self=L_self, label=label)


def _cell_centre_points(nx, ny, pitch, z):
    xs = [(i - (nx - 1) / 2.0) * pitch for j in range(ny) for i in range(nx)]
    ys = [(j - (ny - 1) / 2.0) * pitch for j in range(ny) for i in range(nx)]
    return np.array(xs), np.array(ys), np.full(nx * ny, z)


def _concat_points(*pts):
    return tuple(np.concatenate([p[i] for p in pts]) for i in range(3))


# ---------------------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------------------
def single_loop(seed: int = 0, n_cfg: int = 1, n_freq: int = 101, grid: int = 32) -> Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    a, rw = 0.050, 0.001
    loops = [circular_loop(a, 64)]
    omega = 2 * np.pi * np.linspace(60 * MHZ, 68 * MHZ, n_freq)
    pts = grid_plane(grid, 0.100, 0.020)
    q = [grid // 4, grid - 1 - grid // 4]
    loss_idx = [iy * grid + ix for iy in q for ix in q]
    st = _structure_from(loops, pts, omega, 0.1, loss_idx,
                         L_self=np.array([circular_loop_inductance(a, rw)]), label="single_loop")
    C = rng.uniform(20 * PF, 200 * PF, size=(n_cfg, 1))
    return Workload("single_loop", [st], C, rw, target_rule=("field_at_C", 100 * PF),
                    meta=dict(seed=seed))


def loop_sweep(n_init: int = 100, n_target: int = 100, grid: int = 32,
               c_init_pf=(0.1, 30.0), c_target_pf=(5.0, 30.0)) -> Workload:
    """Initialisation sweep on the single loop at 63.6 MHz (the paper's Sec. V-A study:
    100 initial capacitances x 100 targets): configuration i * n_target + j starts from the
    i-th initial value and fits the field made by the j-th target capacitance
    (target_rule "field_at_C_per_cfg": the caller evaluates the forward map there)."""
    a, rw = 0.050, 0.001
    loops = [circular_loop(a, 64)]
    omega = 2 * np.pi * np.array([63.6 * MHZ])
    pts = grid_plane(grid, 0.100, 0.020)
    q = [grid // 4, grid - 1 - grid // 4]
    loss_idx = [iy * grid + ix for iy in q for ix in q]
    st = _structure_from(loops, pts, omega, 0.1, loss_idx,
                         L_self=np.array([circular_loop_inductance(a, rw)]), label="loop_sweep")
    c0 = np.linspace(c_init_pf[0], c_init_pf[1], n_init) * PF
    ct = np.linspace(c_target_pf[0], c_target_pf[1], n_target) * PF
    C = np.repeat(c0, n_target)[:, None]
    Ct = np.tile(ct, n_init)[:, None]
    return Workload("loop_sweep", [st], C, rw, target_rule=("field_at_C_per_cfg", Ct),
                    target_per_cfg=True, meta=dict(n_init=n_init, n_target=n_target))


def circle_array(nx: int = 3, ny: int = 3, seed: int = 0, n_cfg: int = 64, n_freq: int = 3,
                 radius: float = 0.025, pitch: float = 0.055, n_seg: int = 64,
                 grid: int = 24, closed_form_L: bool = True) -> Workload:
    """An nx x ny array of circular loops (regular n_seg-gons of the given radius); the
    mutual inductances couple oblique segment pairs; the self inductances take the
    closed-form loop value, or (closed_form_L=False) come from the polygon's own segment
    pairs, corners included."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rw = 0.001
    loops = [circular_loop(radius, n_seg, (i - (nx - 1) / 2.0) * pitch, (j - (ny - 1) / 2.0) * pitch)
             for j in range(ny) for i in range(nx)]
    omega = 2 * np.pi * np.linspace(60 * MHZ, 68 * MHZ, n_freq)
    hx, hy = (nx + 1) * pitch / 2.0, (ny + 1) * pitch / 2.0
    pts = _concat_points(grid_plane(grid, hx, 0.020, half_span_y=hy),
                         _cell_centre_points(nx, ny, pitch, 0.040))
    loss_idx = np.arange(grid * grid, grid * grid + nx * ny)
    Ls = np.full(nx * ny, circular_loop_inductance(radius, rw)) if closed_form_L else None
    st = _structure_from(loops, pts, omega, 0.1, loss_idx, L_self=Ls, label=f"circles_{nx}x{ny}")
    C = rng.uniform(20 * PF, 200 * PF, size=(n_cfg, nx * ny))
    target = rng.standard_normal(n_freq * nx * ny) * 1e-6
    return Workload(f"circles_{nx}x{ny}", [st], C, rw, target=target, meta=dict(seed=seed))


def line_8x1(seed: int = 0, n_cfg: int = 1024, n_freq: int = 201, grid: int = 64) -> Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    loops = square_array(8, 1)
    omega = 2 * np.pi * np.linspace(60 * MHZ, 68 * MHZ, n_freq)
    pts = _concat_points(grid_plane(grid, 0.250, 0.020), _cell_centre_points(8, 1, 0.055, 0.040))
    loss_idx = np.arange(grid * grid, grid * grid + 8)
    st = _structure_from(loops, pts, omega, 0.1, loss_idx, label="line_8x1")
    C = rng.uniform(20 * PF, 200 * PF, size=(n_cfg, 8))
    return Workload("line_8x1", [st], C, 0.001, target_rule=("field_at_C", 50 * PF),
                    meta=dict(seed=seed))


def array_8x8(seed: int = 0, n_cfg: int = 4096, grid: int = 128, planes=(0.010, 0.020, 0.030, 0.040),
              freqs_hz=(63.6 * MHZ,)) -> Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    loops = square_array(8, 8)
    omega = 2 * np.pi * np.asarray(freqs_hz, float)
    pts = _concat_points(*[grid_plane(grid, 0.250, z) for z in planes],
                         _cell_centre_points(8, 8, 0.055, 0.040))
    n_grid = grid * grid * len(planes)
    loss_idx = np.arange(n_grid, n_grid + 64)
    st = _structure_from(loops, pts, omega, 0.1, loss_idx, label="array_8x8")
    C = rng.uniform(20 * PF, 200 * PF, size=(n_cfg, 64))
    target = rng.standard_normal(len(omega) * 64) * 1e-6
    return Workload("array_8x8", [st], C, 0.001, target=target, meta=dict(seed=seed))


RAGGED_SHAPES = {1: (1, 1), 8: (8, 1), 16: (4, 4), 32: (8, 4), 64: (8, 8), 128: (16, 8)}


def ragged(seed: int = 0, n_struct: int = 10000, grid: int = 64, max_freq: int = 16,
           port_choices=(1, 8, 16, 32, 64, 128)) -> Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = rng.choice(np.asarray(port_choices), size=n_struct)
    nf = rng.integers(1, max_freq + 1, size=n_struct)
    structs = []
    for s in range(n_struct):
        nx, ny = RAGGED_SHAPES[int(ns[s])]
        loops = square_array(nx, ny)
        f = np.sort(rng.uniform(60 * MHZ, 68 * MHZ, size=int(nf[s])))
        hx, hy = (nx + 1) * 0.055 / 2.0, (ny + 1) * 0.055 / 2.0
        pts = _concat_points(grid_plane(grid, hx, 0.020, half_span_y=hy),
                             _cell_centre_points(nx, ny, 0.055, 0.040))
        loss_idx = np.arange(grid * grid, grid * grid + nx * ny)
        structs.append(_structure_from(loops, pts, 2 * np.pi * f, 0.1, loss_idx,
                                       label=f"ragged_{nx}x{ny}"))
    n_total = sum(st.n_ports for st in structs)
    C = rng.uniform(20 * PF, 200 * PF, size=(1, n_total))
    n_t = sum(st.n_freq * st.n_loss for st in structs)
    target = rng.standard_normal(n_t) * 1e-6
    return Workload("ragged", structs, C, 0.001, target=target, meta=dict(seed=seed))


def array_32x32(seed: int = 0, n_cfg: int = 256, grid: int = 512,
                planes=(0.010, 0.020, 0.030, 0.040), seg_per_side: int = 16) -> Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    loops = square_array(32, 32, seg_per_side=seg_per_side)
    omega = 2 * np.pi * np.array([63.6 * MHZ])
    pts = _concat_points(*[grid_plane(grid, 0.900, z) for z in planes],
                         _cell_centre_points(32, 32, 0.055, 0.040))
    n_grid = grid * grid * len(planes)
    loss_idx = np.arange(n_grid, n_grid + 1024)
    st = _structure_from(loops, pts, omega, 0.1, loss_idx, label="array_32x32")
    C = rng.uniform(20 * PF, 200 * PF, size=(n_cfg, 1024))
    target = rng.standard_normal(1024) * 1e-6
    return Workload("array_32x32", [st], C, 0.001, target=target, meta=dict(seed=seed))


def random_cotangent(shape, seed: int = 1) -> np.ndarray:
    """Seeded complex field cotangent dL/dRe B + j dL/dIm B for backward tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@dataclass
class SrouteWorkload:
    """Inputs of the scattering-parameter route (one structure)."""
    name: str
    S0: np.ndarray        # complex [F, n0, n0]
    field: np.ndarray     # complex [F, P, n0]
    sc_const: np.ndarray  # complex [F, n, n], n = n0 + n1
    rows: np.ndarray      # int32 [nS]: the loads' positions in S_C (diagonal of S11)
    cols: np.ndarray
    n1: int
    omega: np.ndarray     # [F] rad/s
    R: np.ndarray         # [n_cfg, nS] ohm (series RC loads)
    C: np.ndarray         # [n_cfg, nS] farad
    Z0: float
    loss_idx: np.ndarray  # int64 [L]
    target: np.ndarray    # real [F, n1, L]

    @property
    def n_cfg(self) -> int:
        return self.C.shape[0]


def sroute_array(nx: int = 8, ny: int = 8, seed: int = 0, n_cfg: int = 4096, grid: int = 128,
                 planes=(0.010, 0.020, 0.030, 0.040), freqs_hz=(63.6 * MHZ,), rho=(0.5, 0.99),
                 Z0: float = 50.0) -> SrouteWorkload:
    """S-route inputs: nx*ny cell ports plus a drive port (n0 = nx ny + 1), one external port.
    S0 = Q diag(rho_k e^{j phi_k}) Q^T with Q a random orthogonal matrix and rho_k in `rho`
    (symmetric: reciprocal; spectral norm < 1: passive). The field of port k is the Bz of a
    z-directed dipole at the port's cell centre (the drive port's at the array centre, 30 mm
    below) times a random complex amplitude, about 1e-6 T per unit wave at 40 mm. Loads:
    R = 0.1 ohm, C ~ U[20, 200] pF; targets |N(0,1)| x 1e-6 T at the 64-style loss points
    above the cell centres."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_cells = nx * ny
    n0, n1 = n_cells + 1, 1
    omega = 2 * np.pi * np.asarray(freqs_hz, float)
    F = len(omega)
    pts = _concat_points(*[grid_plane(grid, 0.250, z) for z in planes],
                         _cell_centre_points(nx, ny, 0.055, 0.040))
    px, py, pz = pts
    n_grid = grid * grid * len(planes)
    loss_idx = np.arange(n_grid, n_grid + n_cells, dtype=np.int64)
    cx, cy, _ = _cell_centre_points(nx, ny, 0.055, 0.0)
    sx = np.append(cx, 0.0)
    sy = np.append(cy, 0.0)
    sz = np.append(np.zeros(n_cells), -0.030)
    dx = px[:, None] - sx[None, :]
    dy = py[:, None] - sy[None, :]
    dz = pz[:, None] - sz[None, :]
    r2 = dx * dx + dy * dy + dz * dz + 1e-4  # 10 mm core
    dip = (3 * dz * dz - r2) / r2 ** 2.5  # z-dipole Bz shape
    scale = 1e-6 / (2.0 / 0.040 ** 3)
    S0 = np.zeros((F, n0, n0), complex)
    field = np.zeros((F, len(px), n0), complex)
    for f in range(F):
        Q, _ = np.linalg.qr(rng.standard_normal((n0, n0)))
        lam = rng.uniform(rho[0], rho[1], n0) * np.exp(1j * rng.uniform(-np.pi, np.pi, n0))
        S0[f] = (Q * lam[None, :]) @ Q.T
        amp = rng.uniform(0.5, 1.5, n0) * np.exp(1j * rng.uniform(-np.pi, np.pi, n0))
        field[f] = dip * (scale * amp)[None, :]
    sc_const = np.zeros((F, n0 + n1, n0 + n1), complex)
    sc_const[:, n0 - 1, n0] = 1.0  # matched source into the drive port
    rows = np.arange(n_cells, dtype=np.int32)
    R = np.full((n_cfg, n_cells), 0.1)
    C = rng.uniform(20 * PF, 200 * PF, size=(n_cfg, n_cells))
    target = np.abs(rng.standard_normal((F, n1, n_cells))) * 1e-6
    return SrouteWorkload(f"sroute_{nx}x{ny}", S0, field, sc_const, rows, rows.copy(), n1, omega,
                          R, C, Z0, loss_idx, target)
