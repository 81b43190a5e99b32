"""Seeded synthetic inputs shaped like the paper's workloads.

Shared by the CUDA path (bench, tests) and by the oracle.  It holds none of
the method's arithmetic: only random initial fields and the workload
definitions, whose parameters are plain numbers (physical inputs where the
paper derives lattice values from them; each side converts them with its own
similarity helper).

Node index is x + nx*(y + ny*z); vector fields have shape (D, N).
"""
import numpy as np

CS2_PK = 1.0 / 3.0  # kinematic pressure of the reference state (eps_g = 1)

# Boundary codes (same meaning on both sides).
PERIODIC, WALL, INLET, OUTLET = 0, 1, 2, 3

# Physical inputs of the drag relation used by the workloads (Sec. 3.6, TEST #4):
# drag coefficient, gravity, lattice speed.
C_D = 0.66
G_PHYS = 9.81
C_LATTICE = 69.2


def _common_physics(R=1000.0):
    """R = 1000, dynamic viscosity ratio 50 (nu_g = 20 nu_l), CGW drag with a
    1 mm dispersed diameter, (R-1) g_hat = 1e-6, stabilisers gamma = 1,
    n_gamma = 200 (the settings of TEST #3/#4)."""
    return dict(
        R=R, omega_g=0.6, nu_ratio_g_over_l=20.0, omega_alpha=1.5, psi_g=0.0, psi_l=0.0,
        drag_model=1, d_m=1.0e-3, C_d=C_D, g_phys=G_PHYS, c_lattice=C_LATTICE,
        g_hat=1.0e-6 / (R - 1.0), gamma=1.0, n_gamma=200, spalding_mode=2, alpha_floor=1e-8,
    )


WORKLOADS = {
    # 1D gas-liquid column, D1Q3, FP64, walls at both ends, gravity along x.
    "column1d": dict(
        lattice="D1Q3", dims=(512, 1, 1), steps=10000, precision="fp64",
        physics=dict(_common_physics(), wall_friction=True, g_axis=0,
                     bc_lo=(WALL, 0, 0), bc_hi=(WALL, 0, 0)),
    ),
    # 2D bubble-column box, D2Q9, FP32, periodic x, walls y, bottom inlet strip.
    "box2d": dict(
        lattice="D2Q9", dims=(512, 2048, 1), steps=20000, precision="fp32",
        physics=dict(_common_physics(), wall_friction=False, g_axis=1,
                     bc_lo=(PERIODIC, INLET, 0), bc_hi=(PERIODIC, WALL, 0),
                     inlet_lo=192, inlet_hi=320, in_alpha=(0.01, 0.3), in_ug=(4.3e-4, 4.3e-3),
                     in_ul=(0.0, 0.0), inlet_ul_mode=1, ramp_nt=1667),
    ),
    # surrogate workload: closed 2D box (periodic x, walls y), D2Q9 FP32, gas
    # plumes at random places (fields_plumes), R = 1000, snapshots every 64 steps
    "surrogate2d": dict(
        lattice="D2Q9", dims=(256, 1024, 1), steps=4096, precision="fp32",
        physics=dict(_common_physics(), wall_friction=False, g_axis=1,
                     bc_lo=(PERIODIC, WALL, 0), bc_hi=(PERIODIC, WALL, 0)),
    ),
    # surrogate workload with the 2D box's inlet: the box2d physics at 256 x
    # 1024, its bottom strip scaled to width 64 (centred), injecting gas at
    # fraction 0.3 and the box's full inlet velocity from the start (no
    # ramp); walls on top, periodic x; initial gas plumes at random places
    "surrogate2d_inlet": dict(
        lattice="D2Q9", dims=(256, 1024, 1), steps=4096, precision="fp32",
        physics=dict(_common_physics(), wall_friction=False, g_axis=1,
                     bc_lo=(PERIODIC, INLET, 0), bc_hi=(PERIODIC, WALL, 0),
                     inlet_lo=96, inlet_hi=160, in_alpha=(0.3, 0.3), in_ug=(4.3e-3, 4.3e-3),
                     in_ul=(0.0, 0.0), inlet_ul_mode=1, ramp_nt=0),
    ),
    # batched sweep: 256 independent D2Q9 columns (see batch_sweep), FP32
    "batch256": dict(lattice="D2Q9", dims=None, steps=10000, precision="fp32", physics=None),
    # 3D column, D3Q19, walls on the four x/y faces, periodic z, gravity along z.
    "column3d": dict(
        lattice="D3Q19", dims=(256, 256, 512), steps=5000, precision="fp16dev",
        physics=dict(_common_physics(), wall_friction=False, g_axis=2,
                     bc_lo=(WALL, WALL, PERIODIC), bc_hi=(WALL, WALL, PERIODIC)),
    ),
}


def batch_sweep(n=256, seed=4, side=(64, 512), R=(10.0, 1000.0), d_mm=(0.5, 5.0)):
    """Parameter sweep of independent 2D D2Q9 columns (batched workload): side
    nx uniform in `side`, ny = 4 nx, density ratio log-uniform in `R`,
    dispersed diameter uniform in `d_mm` (mm), (R-1) g_hat = 1e-6, gamma = 1,
    n_gamma = 200, periodic x, walls y, gravity along y, FP32.  Returns a
    list of (dims, physics) with physics in the form of the other workloads."""
    r = rng(seed)
    out = []
    for i in range(n):
        nx = int(r.integers(side[0], side[1] + 1))
        Ri = float(np.exp(r.uniform(np.log(R[0]), np.log(R[1]))))
        d = float(r.uniform(d_mm[0], d_mm[1])) * 1e-3
        ph = dict(_common_physics(Ri), d_m=d, wall_friction=False, g_axis=1,
                  bc_lo=(PERIODIC, WALL, 0), bc_hi=(PERIODIC, WALL, 0))
        out.append(((nx, 4 * nx, 1), ph))
    return out


def surrogate_inlet(seed, nx=256, width=64, alpha=(0.2, 0.4), u_scale=(0.5, 1.0)):
    """Physics of one trajectory of the surrogate's inlet recipe: the
    "surrogate2d_inlet" workload with its inlet varied by seed: the strip
    (width `width`) at a uniform position along x, the injected gas fraction
    uniform in `alpha`, the gas velocity the box's full inlet velocity times
    a factor uniform in `u_scale`."""
    r = rng(seed)
    base = WORKLOADS["surrogate2d_inlet"]["physics"]
    x0 = int(r.integers(0, nx - width + 1))
    a_in = float(r.uniform(*alpha))
    u_in = float(r.uniform(*u_scale)) * base["in_ug"][1]
    return dict(base, inlet_lo=x0, inlet_hi=x0 + width, in_alpha=(a_in, a_in), in_ug=(u_in, u_in))


def fields_step_profile(nx, ny, seed, low=0.9, high=0.1, noise=1e-3):
    """alpha_g = `low` below mid-height, `high` above, plus U(-noise, noise);
    at rest; p_k at the reference value."""
    r = rng(seed)
    n = nx * ny
    y = np.arange(n) // nx
    a = np.where(y < ny // 2, low, high) + r.uniform(-noise, noise, n)
    z = np.zeros((2, n))
    return dict(alpha_g=np.clip(a, 0.01, 0.99), u_g=z.copy(), u_l=z.copy(), p_k=np.full(n, CS2_PK))


def fields_smooth1d(n, eps, U=0.64):
    """Smooth periodic 1D state for convergence studies, cell-centred nodes
    x_i = (i + 1/2)/n of the unit interval: alpha_g = 0.3 + 0.05 sin(2 pi x),
    u_g = eps U sin(2 pi x + 0.3) (a lattice velocity: continuum U times the
    mesh spacing eps), u_l with zero mixture flux alpha_g u_g + alpha_l u_l = 0
    (the 1D divergence-free state), p_k uniform at the reference value."""
    x = (np.arange(n) + 0.5) / n
    a = 0.3 + 0.05 * np.sin(2.0 * np.pi * x)
    ug = eps * U * np.sin(2.0 * np.pi * x + 0.3)
    ul = -a * ug / (1.0 - a)
    return dict(alpha_g=a, u_g=ug[None, :], u_l=ul[None, :], p_k=np.full(n, CS2_PK))


def fields_smooth2d(n, eps, U=0.64):
    """Smooth doubly periodic 2D state on the unit square (cell-centred n x n
    nodes): alpha_g = 0.3 + 0.05 sin(2 pi x) sin(2 pi y), both phases in the
    divergence-free Taylor-Green field eps U (sin 2 pi x cos 2 pi y,
    -cos 2 pi x sin 2 pi y) (so the mixture flux is divergence-free), p_k
    uniform.  Vector fields (2, n*n), x fastest."""
    c = (np.arange(n) + 0.5) / n
    y, x = np.meshgrid(c, c, indexing="ij")
    a = (0.3 + 0.05 * np.sin(2.0 * np.pi * x) * np.sin(2.0 * np.pi * y)).reshape(-1)
    u = eps * U * np.stack([np.sin(2.0 * np.pi * x) * np.cos(2.0 * np.pi * y),
                            -np.cos(2.0 * np.pi * x) * np.sin(2.0 * np.pi * y)]).reshape(2, -1)
    return dict(alpha_g=a, u_g=u.copy(), u_l=u.copy(), p_k=np.full(n * n, CS2_PK))


def fields_plumes(nx, ny, seed, background=0.02, blobs=(3, 7), amp=(0.15, 0.4), radius=(8.0, 24.0)):
    """Gas plumes in a liquid column: alpha_g = background plus Gaussian blobs
    (count uniform in `blobs`, amplitude in `amp`, radius in `radius` nodes)
    centred at random x and in the lower half of y, clipped to [0.01, 0.6];
    both phases at rest plus U(-1e-5, 1e-5) velocity noise; p_k reference."""
    r = rng(seed)
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    a = np.full((ny, nx), background)
    for _ in range(int(r.integers(blobs[0], blobs[1] + 1))):
        xc, yc = r.uniform(0, nx), r.uniform(0.1 * ny, 0.5 * ny)
        rad, am = r.uniform(*radius), r.uniform(*amp)
        dx = np.minimum(np.abs(x - xc), nx - np.abs(x - xc))  # periodic in x
        a = a + am * np.exp(-(dx ** 2 + (y - yc) ** 2) / (2.0 * rad ** 2))
    n = nx * ny
    return dict(alpha_g=np.clip(a, 0.01, 0.6).reshape(-1), u_g=r.uniform(-1e-5, 1e-5, (2, n)),
                u_l=r.uniform(-1e-5, 1e-5, (2, n)), p_k=np.full(n, CS2_PK))


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def fields_column1d(n=512, seed=1):
    """alpha_g = 0.9 below mid-column, 0.1 above, plus U(-1e-3, 1e-3), clipped to
    [0.01, 0.99]; both phases at rest; p_k at the reference value."""
    r = rng(seed)
    a = np.where(np.arange(n) < n // 2, 0.9, 0.1) + r.uniform(-1e-3, 1e-3, n)
    a = np.clip(a, 0.01, 0.99)
    z = np.zeros((1, n))
    return dict(alpha_g=a, u_g=z.copy(), u_l=z.copy(), p_k=np.full(n, CS2_PK))


def fields_box2d(nx=512, ny=2048, seed=2, alpha0=0.01, u_noise=4.3e-5):
    """Background alpha_g = 0.01; every velocity component of both phases is
    U(-1, 1) * 1 % of the maximum inlet gas velocity."""
    r = rng(seed)
    n = nx * ny
    return dict(alpha_g=np.full(n, alpha0),
                u_g=r.uniform(-1.0, 1.0, (2, n)) * u_noise,
                u_l=r.uniform(-1.0, 1.0, (2, n)) * u_noise,
                p_k=np.full(n, CS2_PK))


def fields_column3d(nx=256, ny=256, nz=512, seed=3, mean=0.05, std=0.01, corr=8.0):
    """alpha_g = mean + std * (white noise smoothed by a Gaussian of standard
    deviation `corr` nodes, periodic FFT filter, re-standardised); at rest."""
    r = rng(seed)
    noise = r.standard_normal((nz, ny, nx))
    k = [np.fft.fftfreq(m) for m in (nz, ny, nx)]
    kz, ky, kx = np.meshgrid(*k, indexing="ij")
    filt = np.exp(-2.0 * (np.pi * corr) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    sm = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))
    sm = (sm - sm.mean()) / sm.std()
    a = np.clip(mean + std * sm, 0.01, 0.99).reshape(-1)
    n = nx * ny * nz
    z = np.zeros((3, n))
    return dict(alpha_g=a, u_g=z.copy(), u_l=z.copy(), p_k=np.full(n, CS2_PK))


def fields_random(D, dims, seed, alpha=(0.2, 0.8), u_amp=2e-3, pk_amp=1e-4):
    """Generic random smooth-ish state for parity tests: alpha_g uniform in
    `alpha`, velocities uniform in +-u_amp, p_k = 1/3 + uniform +-pk_amp."""
    r = rng(seed)
    n = int(np.prod(dims))
    return dict(alpha_g=r.uniform(alpha[0], alpha[1], n),
                u_g=r.uniform(-u_amp, u_amp, (D, n)),
                u_l=r.uniform(-u_amp, u_amp, (D, n)),
                p_k=CS2_PK + r.uniform(-pk_amp, pk_amp, n))


def fields_for(name, dims=None, seed=None):
    w = WORKLOADS[name]
    dims = dims or w["dims"]
    if name == "column1d":
        return fields_column1d(dims[0], seed if seed is not None else 1)
    if name == "box2d":
        return fields_box2d(dims[0], dims[1], seed if seed is not None else 2)
    if name == "column3d":
        return fields_column3d(dims[0], dims[1], dims[2], seed if seed is not None else 3)
    raise KeyError(name)
