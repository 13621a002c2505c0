"""Named synthetic workloads with the shapes of the paper's experiments.

The paper's geometries (Sec. 5.2-5.4) are not shipped with it; these seeded
synthetic problems stand in for them:

  square65_hh  65 x 65 P1 triangles on [0,1]^2 cm, sigma = 1 mS/cm, HH,
               50 uA/cm^2 for t <= 1 ms on the 0.1 cm corner, dt 0.05, T 20 ms.
  slab_ttp     201 x 71 x 31 Kuhn tets on a 2.0 x 0.7 x 0.3 cm slab,
               D = diag(1.33, 0.18, 0.18) mS/cm (fibres along x), TTP06 epi,
               50 uA/cm^2 for t <= 2 ms on the 0.15 cm corner cube, dt 0.05,
               T 50 ms (the 3-D cuboid of Sec. 5.3 at 0.1 mm).
  shell_ttp    32 x 362 x 362 structured box mapped onto a truncated prolate-
               ellipsoidal shell (semi-axes 5/2.5 cm outer, 4.3/1.8 cm inner,
               cut at z = 2 cm; ~4.2 M nodes, ~24 M Kuhn tets, interior nodes
               jittered by +-20% of the local spacing), fibre angle +60 deg
               (endo) -> -60 deg (epi), TTP06, apical stimulus, dt 0.05,
               T 100 ms.

Tissue constants follow Table 1 in centimetres: chi = 1400 /cm, Cm = 1 uF/cm^2.
Ionic model ids: 0 none (pure diffusion), 1 passive test model, 2 Hodgkin-
Huxley, 3 ten Tusscher-Panfilov 2006 epicardial.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .fields import axis_D, corner_mask, fibre_D, fibrosis_D, isotropic_D, radius_mask
from .meshes import line_mesh, shell_tet_mesh, slab_tet_mesh, square_tri_mesh

MODEL_NONE, MODEL_PASSIVE, MODEL_HH, MODEL_TTP06 = 0, 1, 2, 3
MODEL_NAMES = {0: "none", 1: "passive", 2: "hh", 3: "ttp06_epi"}


@dataclass
class Workload:
    name: str
    coords: np.ndarray
    cells: np.ndarray
    D: np.ndarray  # (n_cells, dim, dim) mS/cm
    model: int
    stim_mask: np.ndarray  # uint8 per node
    stim_amp: float = 50.0  # uA/cm^2
    t_on: float = 0.0
    t_off: float = 1.0
    dt: float = 0.05
    T: float = 20.0
    chi: float = 1400.0
    Cm: float = 1.0
    rho_every: int = 1  # 0 = once at start
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.coords.shape[0]

    @property
    def dim(self) -> int:
        return self.coords.shape[1]

    @property
    def steps(self) -> int:
        return int(round(self.T / self.dt))


def _square(nx, ny, lx, ly, model, sigma=1.0, corner=0.1, t_off=1.0, dt=0.05, T=20.0, name=None):
    coords, cells = square_tri_mesh(nx, ny, lx, ly)
    D = isotropic_D(cells.shape[0], 2, sigma)
    return Workload(name or f"square{nx}x{ny}", coords, cells, D, model,
                    corner_mask(coords, corner), t_off=t_off, dt=dt, T=T)


def _slab(nx, ny, nz, lx, ly, lz, model, sig=(1.33, 0.18, 0.18), corner=0.15,
          t_off=2.0, dt=0.05, T=50.0, name=None):
    coords, cells = slab_tet_mesh(nx, ny, nz, lx, ly, lz)
    D = axis_D(cells.shape[0], sig)
    return Workload(name or f"slab{nx}x{ny}x{nz}", coords, cells, D, model,
                    corner_mask(coords, corner), t_off=t_off, dt=dt, T=T, rho_every=0)


def shell_fibres(coords, cells, param):
    """Cell fibre vectors: angle +60 deg at r=0 (endo) to -60 deg at r=1 (epi)
    in the (e_phi, e_theta) tangent plane, evaluated at the cell centroid."""
    pr, rs_in, rl_in, thick, z_top = param
    c = coords[cells].mean(axis=1)
    rc = pr[cells].mean(axis=1)
    phi = np.arctan2(c[:, 1], c[:, 0])
    e_phi = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], axis=1)
    # e_theta: derivative of the surface point along theta at fixed r, normalised
    rs = rs_in + thick * rc
    rl = rl_in + thick * rc
    rho_xy = np.hypot(c[:, 0], c[:, 1])
    sin_t = np.clip(rho_xy / rs, 0.0, 1.0)
    cos_t = np.clip(c[:, 2] / rl, -1.0, 1.0)
    e_th = np.stack([rs * cos_t * np.cos(phi), rs * cos_t * np.sin(phi), -rl * sin_t], axis=1)
    e_th /= np.linalg.norm(e_th, axis=1, keepdims=True)
    alpha = np.deg2rad(60.0 * (1.0 - rc) - 60.0 * rc)
    return np.cos(alpha)[:, None] * e_phi + np.sin(alpha)[:, None] * e_th


def make_workload(name: str, **kw) -> Workload:
    """Build a named workload; keyword arguments override the defaults."""
    if name == "square65_hh":
        w = _square(65, 65, 1.0, 1.0, MODEL_HH, name=name)
        w.rho_every = 1
    elif name == "slab_ttp":
        w = _slab(201, 71, 31, 2.0, 0.7, 0.3, MODEL_TTP06, name=name)
    elif name == "slab_hh":
        w = _slab(201, 71, 31, 2.0, 0.7, 0.3, MODEL_HH, name=name)
    elif name == "shell_ttp":
        nr = kw.pop("nr", 32)
        nuv = kw.pop("nuv", 362)
        coords, cells, param = shell_tet_mesh(nr, nuv, return_param=True)
        a_l = shell_fibres(coords, cells, param)
        D = fibre_D(a_l, 1.33, 0.18)
        rl_out = param[2] + param[3]
        w = Workload(name, coords, cells, D, MODEL_TTP06,
                     radius_mask(coords, (0.0, 0.0, -rl_out), 0.3),
                     t_off=2.0, dt=0.05, T=100.0, rho_every=0)
    elif name == "cable_ttp":
        # Sec. 5.1 practical-stability set-up: [0, 2] cm at dx = 0.0025 cm (801
        # nodes), sigma = 1.33 mS/cm, TTP06, stimulus on x <= 0.15 cm for
        # t <= 2 ms, T = 100 ms
        coords, cells = line_mesh(801, 2.0)
        w = Workload(name, coords, cells, isotropic_D(cells.shape[0], 1, 1.33), MODEL_TTP06,
                     (coords[:, 0] <= 0.15 + 1e-12).astype(np.uint8), t_off=2.0, dt=0.05, T=100.0,
                     rho_every=0)
    elif name.startswith("fibslab"):
        # slab with fibrosis: fibres along x (sigma_l 1.33, sigma_t 0.18) and
        # sigma_t = 0 where a seeded smooth random field (correlation length
        # 0.05 cm) exceeds its median
        dims, model = name[len("fibslab"):].split("_")
        nx, ny, nz = (int(v) for v in dims.split("x"))
        h = kw.pop("h", 0.01)
        seed = kw.pop("seed", 11)
        mid = {"hh": MODEL_HH, "ttp": MODEL_TTP06, "none": MODEL_NONE, "passive": MODEL_PASSIVE}[model]
        w = _slab(nx, ny, nz, (nx - 1) * h, (ny - 1) * h, (nz - 1) * h, mid, name=name)
        a_l = np.tile(np.array([1.0, 0.0, 0.0]), (w.cells.shape[0], 1))
        w.D, fib = fibrosis_D(w.coords, w.cells, a_l, 1.33, 0.18, seed, 0.05)
        w.extra["fibrotic_cells"] = fib
    elif name.startswith("square"):
        # squareNxM_model, e.g. square17x17_hh on [0, (N-1)h] with h from kw
        dims, model = name[len("square"):].split("_")
        nx, ny = (int(v) for v in dims.split("x"))
        h = kw.pop("h", 1.0 / 64)
        mid = {"hh": MODEL_HH, "ttp": MODEL_TTP06, "none": MODEL_NONE, "passive": MODEL_PASSIVE}[model]
        w = _square(nx, ny, (nx - 1) * h, (ny - 1) * h, mid, name=name)
    elif name.startswith("slab"):
        dims, model = name[len("slab"):].split("_")
        nx, ny, nz = (int(v) for v in dims.split("x"))
        h = kw.pop("h", 0.01)
        mid = {"hh": MODEL_HH, "ttp": MODEL_TTP06, "none": MODEL_NONE, "passive": MODEL_PASSIVE}[model]
        w = _slab(nx, ny, nz, (nx - 1) * h, (ny - 1) * h, (nz - 1) * h, mid, name=name)
    elif name.startswith("line"):
        n, model = name[len("line"):].split("_")
        n = int(n)
        length = kw.pop("length", 1.0)
        coords, cells = line_mesh(n, length)
        mid = {"hh": MODEL_HH, "ttp": MODEL_TTP06, "none": MODEL_NONE, "passive": MODEL_PASSIVE}[model]
        w = Workload(name, coords, cells, isotropic_D(cells.shape[0], 1, 1.0), mid,
                     corner_mask(coords, 0.1 * length))
    else:
        raise KeyError(f"unknown workload {name!r}")
    for k, v in kw.items():
        if not hasattr(w, k):
            raise KeyError(f"unknown workload field {k!r}")
        setattr(w, k, v)
    return w


WORKLOADS = ("square65_hh", "slab_ttp", "shell_ttp")


def batched_specs(count: int = 256, seed: int = 3, n_min: float = 8e3, n_max: float = 5e5):
    """Specifications of the batched workload (one dict per instance).

    n_i = exp(U(ln n_min, ln n_max)); geometry by coin flip: 2-D square of
    side round(sqrt(n)) nodes (h = 1/64 cm) or 3-D slab with node counts in
    the ratio 20:7:3 (h = 0.01 cm); sigma_l ~ U(0.8, 2.0) mS/cm, anisotropy
    sigma_l/sigma_t ~ U(4, 10), fibres along x; a stimulus patch (radius
    0.1 cm, 50 uA/cm^2 for 2 ms) centred at a boundary node chosen uniformly;
    ionic model HH or TTP06 by coin flip.  All draws come from SplitMix64 on
    (seed, instance, field).
    """
    import math

    from .fields import splitmix64, u01

    def draw(i, f):
        return float(u01(splitmix64(np.uint64(seed), np.uint64((i << 8) | f))))

    out = []
    for i in range(count):
        n = math.exp(math.log(n_min) + draw(i, 0) * (math.log(n_max) - math.log(n_min)))
        is3d = draw(i, 1) < 0.5
        sig_l = 0.8 + 1.2 * draw(i, 2)
        ratio = 4.0 + 6.0 * draw(i, 3)
        model = MODEL_HH if draw(i, 4) < 0.5 else MODEL_TTP06
        if is3d:
            k = (n / 420.0) ** (1.0 / 3.0)
            dims = (max(2, round(20 * k)), max(2, round(7 * k)), max(2, round(3 * k)))
            h = 0.01
        else:
            side = max(2, round(math.sqrt(n)))
            dims = (side, side)
            h = 1.0 / 64
        out.append(dict(index=i, dims=dims, h=h, sigma_l=sig_l, sigma_t=sig_l / ratio, model=model,
                        u_site=draw(i, 5)))
    return out


def batched_workload(spec) -> Workload:
    """Build the mesh and inputs of one batched instance from its spec."""
    dims, h = spec["dims"], spec["h"]
    if len(dims) == 2:
        coords, cells = square_tri_mesh(dims[0], dims[1], (dims[0] - 1) * h, (dims[1] - 1) * h)
        D = axis_D(cells.shape[0], (spec["sigma_l"], spec["sigma_t"]))
    else:
        coords, cells = slab_tet_mesh(*dims, *[(d - 1) * h for d in dims])
        D = axis_D(cells.shape[0], (spec["sigma_l"], spec["sigma_t"], spec["sigma_t"]))
    lo, hi = coords.min(axis=0), coords.max(axis=0)
    boundary = np.nonzero(np.any((np.abs(coords - lo) < 1e-12) | (np.abs(coords - hi) < 1e-12), axis=1))[0]
    site = boundary[min(int(spec["u_site"] * boundary.size), boundary.size - 1)]
    mask = radius_mask(coords, coords[site], 0.1)
    return Workload(f"batch{spec['index']}", coords, cells, D, spec["model"], mask,
                    t_off=2.0, dt=0.05, T=50.0, rho_every=0)


def served_requests(count: int = 100, rate: float = 20.0, seed: int = 4, n_min: float = 1e4,
                    n_max: float = 2e6, horizon=(20.0, 400.0), size_classes: int = 8):
    """Seeded request stream for the served form.

    Poisson arrivals (exponential inter-arrival times of mean 1/rate s); each
    request is a monodomain solve with n ~ log-U(n_min, n_max) nodes, rounded
    to one of ``size_classes`` log-spaced size classes so that meshes can be
    prepared once per class; geometry slab or shell and ionic model HH or
    TTP06 by coin flips; horizon ~ U(horizon) ms at dt = 0.05 ms.
    """
    import math

    from .fields import splitmix64, u01

    def draw(i, f):
        return float(u01(splitmix64(np.uint64(seed), np.uint64((i << 8) | f))))

    classes = np.exp(np.linspace(math.log(n_min), math.log(n_max), size_classes))
    t = 0.0
    out = []
    for i in range(count):
        t += -math.log(max(1e-300, 1.0 - draw(i, 0))) / rate
        n = math.exp(math.log(n_min) + draw(i, 1) * (math.log(n_max) - math.log(n_min)))
        cls = int(np.argmin(np.abs(np.log(classes) - math.log(n))))
        geom = "slab" if draw(i, 2) < 0.5 else "shell"
        model = MODEL_HH if draw(i, 3) < 0.5 else MODEL_TTP06
        hz = horizon[0] + (horizon[1] - horizon[0]) * draw(i, 4)
        steps = max(1, int(round(hz / 0.05)))
        out.append(dict(index=i, arrival=t, n_target=float(classes[cls]), size_class=cls, geometry=geom,
                        model=model, steps=steps))
    return out


def request_workload(req, model=None) -> Workload:
    """Mesh and inputs of one served request (same for every request of its
    geometry and size class; the ionic model is the request's)."""
    n = req["n_target"]
    mid = req["model"] if model is None else model
    if req["geometry"] == "slab":
        k = (n / 420.0) ** (1.0 / 3.0)
        dims = (max(2, round(20 * k)), max(2, round(7 * k)), max(2, round(3 * k)))
        h = 0.01
        coords, cells = slab_tet_mesh(*dims, *[(d - 1) * h for d in dims])
        D = axis_D(cells.shape[0], (1.33, 0.18, 0.18))
        mask = corner_mask(coords, 0.15)
    else:
        nuv = max(4, round((11.0 * n) ** (1.0 / 3.0)))
        nr = max(3, round(n / (nuv * nuv)))
        coords, cells, param = shell_tet_mesh(nr, nuv, return_param=True)
        D = fibre_D(shell_fibres(coords, cells, param), 1.33, 0.18)
        mask = radius_mask(coords, (0.0, 0.0, -(param[2] + param[3])), 0.3)
    return Workload(f"req{req['index']}", coords, cells, D, mid, mask, t_off=2.0, dt=0.05,
                    T=req["steps"] * 0.05, rho_every=0)
