"""Test helpers: run the FP64 oracle over a (possibly ragged) workload, in the layouts of
the C ABI, and relative-error metrics. Expected values come only from oracle/."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2503_18479_gb300 import workloads as W


def rel(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0))


def loss_err(loss, ref, loss_idx) -> float:
    """Error of the objective mean_{f,l} (|B| - t)^2 per configuration, scaled by its
    sensitivity to the field. A field error dB moves the objective by at most
    2 sqrt(loss) rms|dB| + rms|dB|^2, so near a good fit (loss -> 0) the plain relative error
    of the objective is the field's relative error times rms|B| / sqrt(loss); dividing by
    loss + 2 sqrt(loss) rms|B| gives the quantity a relative field tolerance bounds.
    `ref` is the oracle's forward dict (B [n_cfg, F, P], loss [n_cfg])."""
    loss = np.asarray(loss, float).ravel()
    lr = np.asarray(ref["loss"], float).ravel()
    bl = np.abs(ref["B"][:, :, np.asarray(loss_idx)])
    rms = np.sqrt(np.mean(bl.reshape(len(lr), -1) ** 2, axis=1))
    den = lr + 2.0 * np.sqrt(lr) * rms
    return float(np.max(np.abs(loss - lr) / np.where(den > 0, den, 1.0)))


def cosine(a, b) -> float:
    a = np.asarray(a, float).ravel()
    b = np.asarray(b, float).ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def structure_basis(wl: W.Workload, s: int):
    st = wl.structures[s]
    H = oracle.basis(st.loop_vtx_off, st.vx, st.vy, st.vz, st.px, st.py, st.pz, wl.wire_radius,
                     comp=st.pcomp)
    status, M = oracle.inductance(st.loop_vtx_off, st.vx, st.vy, st.vz, wl.wire_radius, st.L_self)
    assert status == 0
    return H, M


def apply_target_rule(wl: W.Workload, bases=None) -> W.Workload:
    """Targets |Bz| at a fixed capacitance (the 'field at C = X' rule), from the oracle."""
    if wl.target is not None or wl.target_rule is None:
        return wl
    kind, c0 = wl.target_rule
    assert kind == "field_at_C"
    blocks = []
    for s, st in enumerate(wl.structures):
        H, M = bases[s] if bases is not None else structure_basis(wl, s)
        C0 = np.full((1, st.n_ports), c0)
        out = oracle.forward(H, M, st.R, C0, st.omega, st.V, want_loss=False)
        blocks.append(np.abs(out["B"][0][:, st.loss_idx]).ravel())
    wl.target = np.concatenate(blocks)
    return wl


def oracle_reference(wl: W.Workload, want_B: bool = True, want_grad: bool = True, cfg=None,
                     gB=None, bases=None):
    """Per-structure oracle results. cfg: optional index array of configurations."""
    res = []
    for s, st in enumerate(wl.structures):
        H, M = bases[s] if bases is not None else structure_basis(wl, s)
        C = wl.structure_C(s)
        if cfg is not None:
            C = C[cfg]
        t = None
        if wl.target is not None:
            t = wl.structure_target(s)
            if wl.target_per_cfg and cfg is not None:
                t = t[cfg]
            if wl.loss_mode == 1:
                t = np.ascontiguousarray(t)
        out = oracle.forward(H, M, st.R, C, st.omega, st.V, st.loss_idx if t is not None else None,
                             t, mode=wl.loss_mode, target_per_cfg=wl.target_per_cfg,
                             want_B=want_B, want_loss=t is not None)
        r = {"H": H, "M": M, "I": out["I"], "B": out["B"], "loss": out["loss"]}
        if want_grad and t is not None:
            r["grad"] = oracle.gradient(H, M, st.R, C, st.omega, st.V, st.loss_idx, t,
                                        mode=wl.loss_mode, target_per_cfg=wl.target_per_cfg)
        if gB is not None:
            r["grad_field"] = oracle.gradient_field(H, M, st.R, C, st.omega, st.V, gB[s])
        res.append(r)
    return res


def split_B(wl: W.Workload, B: np.ndarray):
    """Concatenated [n_cfg, sum F_s P_s] field -> list of [n_cfg, F_s, P_s]."""
    out, o = [], 0
    for st in wl.structures:
        n = st.n_freq * st.n_points
        out.append(B[:, o:o + n].reshape(B.shape[0], st.n_freq, st.n_points))
        o += n
    return out


def split_I(wl: W.Workload, I: np.ndarray):
    out, o = [], 0
    for st in wl.structures:
        n = st.n_freq * st.n_ports
        out.append(I[:, o:o + n].reshape(I.shape[0], st.n_freq, st.n_ports))
        o += n
    return out


def split_ports(wl: W.Workload, G: np.ndarray):
    po = wl.port_off()
    return [G[:, po[s]:po[s + 1]] for s in range(len(wl.structures))]


def small_8x8(n_cfg=200, grid=24, planes=(0.02, 0.04), seed=0):
    return W.array_8x8(seed=seed, n_cfg=n_cfg, grid=grid, planes=planes)


def small_line(n_cfg=96, n_freq=5, grid=20, seed=0):
    wl = W.line_8x1(seed=seed, n_cfg=n_cfg, n_freq=n_freq, grid=grid)
    return apply_target_rule(wl)


def small_loop(n_cfg=16, n_freq=11, grid=16, seed=0):
    wl = W.single_loop(seed=seed, n_cfg=n_cfg, n_freq=n_freq, grid=grid)
    return apply_target_rule(wl)


def small_ragged(n_struct=12, seed=3, grid=12, max_freq=4, ports=(1, 8, 16, 32, 64)):
    return W.ragged(seed=seed, n_struct=n_struct, grid=grid, max_freq=max_freq, port_choices=ports)


def with_components(wl: W.Workload, seed: int) -> W.Workload:
    """The same structures with a seeded field component (0 z, 1 x, 2 y) at every point."""
    import dataclasses
    rng = np.random.Generator(np.random.PCG64(seed))
    ss = [dataclasses.replace(st, pcomp=rng.integers(0, 3, size=st.n_points).astype(np.int8))
          for st in wl.structures]
    return dataclasses.replace(wl, structures=ss)


def small_rect(nx, ny, n_cfg=20, n_freq=2, grid=10, seed=0):
    """An nx x ny array of the standard square cells (any port count), grid at z = 20 mm,
    loss points above the cell centres, random targets."""
    rng = np.random.Generator(np.random.PCG64(seed))
    loops = W.square_array(nx, ny)
    omega = 2 * np.pi * np.linspace(60e6, 68e6, n_freq)
    hx, hy = (nx + 1) * 0.055 / 2.0, (ny + 1) * 0.055 / 2.0
    pts = W._concat_points(W.grid_plane(grid, hx, 0.020, half_span_y=hy),
                           W._cell_centre_points(nx, ny, 0.055, 0.040))
    loss_idx = np.arange(grid * grid, grid * grid + nx * ny)
    st = W._structure_from(loops, pts, omega, 0.1, loss_idx, label=f"rect_{nx}x{ny}")
    C = rng.uniform(20e-12, 200e-12, size=(n_cfg, nx * ny))
    target = rng.standard_normal(n_freq * nx * ny) * 1e-6
    return W.Workload(f"rect_{nx}x{ny}", [st], C, 0.001, target=target, meta=dict(seed=seed))
