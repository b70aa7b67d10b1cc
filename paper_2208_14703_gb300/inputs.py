"""Seeded synthetic inputs for the implicit M1 step.

This module generates the input states, opacities and inflow profiles that the
CUDA path, the tests, the benchmark and the CPU oracle all consume.  It holds
none of the solver's arithmetic: it only draws random numbers and lays out
initial conditions.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) evaluated on a counter, so a
field is a pure function of (seed, index); normals use the Box-Muller
transform.  Opacity fields follow the recipe of the workloads:
log10(sigma) = 1 + 3 g clipped to [-2, 4], g a unit-variance Gaussian random
field (white noise smoothed by a periodic Gaussian filter of correlation length
8 cells), so sigma spans 1e-2 .. 1e4 and optically thin and thick regions mix.

Every case is a dict with keys
  desc:   dim, nx, ny, lx, ly, bc (west, east, south, north), c, a_r, c_v
  dt:     physical time step (CFL * h / c)
  state:  float64 (4, ny, nx) planes E, Fx, Fy, T
  sa, ss: float64 (ny, nx) absorption / scattering opacities
  inflow: float64 (4, 3, max(nx, ny)) prescribed wall states or None
  lmax, tol: the level count and relative residual target of the workload
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n outputs of splitmix64 started at state `seed` (counter form)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """Standard normals by Box-Muller on two counter streams."""
    u1 = uniform(seed * 2 + 1, n)
    u2 = uniform(seed * 2 + 2, n)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def gaussian_field(nx: int, ny: int, seed: int, corr: float = 8.0) -> np.ndarray:
    """Unit-variance, zero-mean Gaussian random field (periodic smoothing by FFT)."""
    w = normal(seed, nx * ny).reshape(ny, nx)
    kx = np.fft.fftfreq(nx)
    ky = np.fft.fftfreq(ny) if ny > 1 else np.zeros(1)
    filt = np.exp(-0.5 * (2 * np.pi * corr) ** 2 * (kx[None, :] ** 2 + ky[:, None] ** 2))
    g = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))
    g -= g.mean()
    s = g.std()
    return g / s if s > 0 else g


def lognormal_opacity(nx: int, ny: int, seed: int, corr: float = 8.0, lo: float = -2.0,
                      hi: float = 4.0) -> np.ndarray:
    g = gaussian_field(nx, ny, seed, corr)
    return 10.0 ** np.clip(1.0 + 3.0 * g, lo, hi)


def _desc(dim, nx, ny, lx, ly, bc, c=1.0, a_r=1.0, c_v=1.0):
    return dict(dim=dim, nx=nx, ny=ny if dim == 2 else 1, lx=lx, ly=ly, bc=list(bc), c=c,
                a_r=a_r, c_v=c_v)


def _state(nx, ny, E, Fx=None, Fy=None, T=None):
    s = np.zeros((4, ny, nx))
    s[0] = E
    if Fx is not None:
        s[1] = Fx
    if Fy is not None:
        s[2] = Fy
    s[3] = 1.0 if T is None else T
    return s


def gaussian_1d(n: int = 256, cfl: float = 50.0, lmax: int = 4, tol: float = 1e-10) -> dict:
    """1D: n cells on [0, 1], c = a_r = C_v = 1, sigma_a = sigma_s = 1, T_g = 1,
    E = 1e-2 + exp(-(x - 0.5)^2 / 0.005), F = 0, periodic, dt = cfl * h / c."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    E = 1e-2 + np.exp(-(x - 0.5) ** 2 / 0.005)
    return dict(desc=_desc(1, n, 1, 1.0, 1.0, ["periodic"] * 4), dt=cfl * h,
                state=_state(n, 1, E[None, :]), sa=np.ones((1, n)), ss=np.ones((1, n)),
                inflow=None, lmax=lmax, tol=tol)


def hot_square_2d(n: int = 1024, cfl: float = 100.0, lmax: int = 8, tol: float = 1e-8,
                  seed_a: int = 1, seed_s: int = 2) -> dict:
    """2D plain-FP64 workload: n x n cells on [0,1]^2, lognormal sigma_a, sigma_s,
    T_g = 1 with a centred hot square of side 1/8 at T_g = 4, E = a_r T_g^4,
    F = 0, reflecting walls, dt = cfl * h / c."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(x, x)
    T = np.where((np.abs(X - 0.5) < 1 / 16) & (np.abs(Y - 0.5) < 1 / 16), 4.0, 1.0)
    return dict(desc=_desc(2, n, n, 1.0, 1.0, ["reflect"] * 4), dt=cfl * h,
                state=_state(n, n, T ** 4, T=T), sa=lognormal_opacity(n, n, seed_a),
                ss=lognormal_opacity(n, n, seed_s), inflow=None, lmax=lmax, tol=tol)


def gaussian_field_3d(nx: int, ny: int, nz: int, seed: int, corr: float = 8.0) -> np.ndarray:
    """Unit-variance, zero-mean Gaussian random field on a periodic 3D grid
    (white noise smoothed by a Gaussian filter by FFT), shape (nz, ny, nx)."""
    w = normal(seed, nx * ny * nz).reshape(nz, ny, nx)
    kx, ky, kz = np.fft.fftfreq(nx), np.fft.fftfreq(ny), np.fft.fftfreq(nz)
    k2 = kx[None, None, :] ** 2 + ky[None, :, None] ** 2 + kz[:, None, None] ** 2
    g = np.real(np.fft.ifftn(np.fft.fftn(w) * np.exp(-0.5 * (2 * np.pi * corr) ** 2 * k2)))
    g -= g.mean()
    s = g.std()
    return g / s if s > 0 else g


def lognormal_opacity_3d(nx: int, ny: int, nz: int, seed: int, corr: float = 8.0,
                         lo: float = -2.0, hi: float = 4.0) -> np.ndarray:
    return 10.0 ** np.clip(1.0 + 3.0 * gaussian_field_3d(nx, ny, nz, seed, corr), lo, hi)


def _desc3(nx, ny, nz, lx, ly, lz, bc, c=1.0, a_r=1.0, c_v=1.0):
    return dict(dim=3, nx=nx, ny=ny, nz=nz, lx=lx, ly=ly, lz=lz, bc=list(bc), c=c, a_r=a_r,
                c_v=c_v)


def hot_cube_3d(n: int = 128, cfl: float = 100.0, lmax: int = 5, tol: float = 1e-8,
                seed_a: int = 21, seed_s: int = 22, bc=("reflect",) * 6) -> dict:
    """3D counterpart of the 2D plain-FP64 workload: n^3 cells on [0,1]^3,
    lognormal sigma_a, sigma_s (the 2D recipe on a 3D random field), T_g = 1 with
    a centred hot cube of side 1/8 at T_g = 4, E = a_r T_g^4, F = 0, reflecting
    walls (x low, x high, y low, y high, z low, z high), dt = cfl * h / c.
    State: float64 (5, n, n, n) planes E, Fx, Fy, Fz, T; opacities (n, n, n)."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    hot = (np.abs(X - 0.5) < 1 / 16) & (np.abs(Y - 0.5) < 1 / 16) & (np.abs(Z - 0.5) < 1 / 16)
    T = np.where(hot, 4.0, 1.0)
    state = np.zeros((5, n, n, n))
    state[0] = T ** 4
    state[4] = T
    return dict(desc=_desc3(n, n, n, 1.0, 1.0, 1.0, bc), dt=cfl * h, state=state,
                sa=lognormal_opacity_3d(n, n, n, seed_a), ss=lognormal_opacity_3d(n, n, n, seed_s),
                inflow=None, lmax=lmax, tol=tol)


def beam_3d(n: int = 32, cfl: float = 100.0, lmax: int = 3, tol: float = 1e-8,
            seed_a: int = 23, seed_s: int = 24) -> dict:
    """3D beam: an f = 1 beam (E = 1, F = (c, 0, 0)) enters through the x-low
    wall into a square channel |y - 1/2|, |z - 1/2| <= 1/16 (sigma = 1e-2) cut
    through the lognormal medium; the rest of that wall holds E = 1, F = 0;
    the other walls reflect.  Background T_g = 1, E = 1, F = 0.  inflow: float64
    (6 walls, 4 fields E, Fx, Fy, Fz, largest face) with the x-low face indexed
    z * n + y."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    chan = np.abs(x - 0.5) <= 1 / 16
    sa = lognormal_opacity_3d(n, n, n, seed_a)
    ss = lognormal_opacity_3d(n, n, n, seed_s)
    box = chan[None, :, None] & chan[:, None, None]          # (z, y, any x)
    box = np.broadcast_to(box, (n, n, n))
    sa[box] = 1e-2
    ss[box] = 1e-2
    face = np.zeros((6, 4, n * n))
    face[0, 0] = 1.0
    face[0, 1] = (chan[:, None] & chan[None, :]).reshape(-1).astype(float)   # (z, y) -> z * n + y
    state = np.zeros((5, n, n, n))
    state[0] = 1.0
    state[4] = 1.0
    return dict(desc=_desc3(n, n, n, 1.0, 1.0, 1.0, ["inflow"] + ["reflect"] * 5), dt=cfl * h,
                state=state, sa=sa, ss=ss, inflow=face, lmax=lmax, tol=tol)


def beam_channel_2d(n: int = 4096, cfl: float = 100.0, lmax: int = 10, tol: float = 1e-8,
                    seed_a: int = 3, seed_s: int = 4) -> dict:
    """2D beam: an f = 1 beam (E = 1, F = (c, 0)) enters through the west wall
    into a thin channel y in [0.45, 0.55] (sigma_a = sigma_s = 1e-2) cut through
    the lognormal medium; the rest of the west wall holds the background state
    (E = 1, F = 0); other walls reflect.  Background T_g = 1, E = 1, F = 0."""
    h = 1.0 / n
    y = (np.arange(n) + 0.5) * h
    chan = (y >= 0.45) & (y <= 0.55)
    sa = lognormal_opacity(n, n, seed_a)
    ss = lognormal_opacity(n, n, seed_s)
    sa[chan, :] = 1e-2
    ss[chan, :] = 1e-2
    inflow = np.zeros((4, 3, n))
    inflow[0, 0, :] = 1.0
    inflow[0, 1, :] = np.where(chan, 1.0, 0.0)
    return dict(desc=_desc(2, n, n, 1.0, 1.0, ["inflow", "reflect", "reflect", "reflect"]),
                dt=cfl * h, state=_state(n, n, np.ones((n, n))), sa=sa, ss=ss, inflow=inflow,
                lmax=lmax, tol=tol)


def paper_beam_2d(n: int = 256, cfl: float = 2000.0, lmax: int = 4, tol: float = 1e-2) -> dict:
    """The beam of Section 4.1 (run in Section 5.1) in nondimensional form.  The
    domain is [-1, 1]^2 with n x n cells; there is no matter (sigma_a = sigma_s
    = 0, the paper's setting); the background is at the radiative temperature
    T_r = 300 K with F = 0, scaled to E = a_r T^4 = 1 (T = 1).  A beam at
    T_r = 1000 K, E = (1000/300)^4, with reduced flux f = 1 at 45 degrees,
    F = c E (1, 1)/sqrt(2), enters through the west wall at y in [-0.875, -0.75].
    The rest of the west wall holds the background state; the other walls
    copy their neighbour (zero-gradient outflow: the paper does not say).
    dt = cfl * h / c with the paper's CFL 2000, so one implicit step reaches the
    steady state; tol = 1e-2 relative residual (Section 5.1)."""
    h = 2.0 / n
    y = -1.0 + (np.arange(n) + 0.5) * h
    beam = (y >= -0.875) & (y <= -0.75)
    e_beam = (1000.0 / 300.0) ** 4
    inflow = np.zeros((4, 3, n))
    inflow[0, 0, :] = np.where(beam, e_beam, 1.0)
    inflow[0, 1, :] = np.where(beam, e_beam / np.sqrt(2.0), 0.0)
    inflow[0, 2, :] = np.where(beam, e_beam / np.sqrt(2.0), 0.0)
    z = np.zeros((n, n))
    return dict(desc=_desc(2, n, n, 2.0, 2.0, ["inflow", "neumann", "neumann", "neumann"]),
                dt=cfl * h, state=_state(n, n, np.ones((n, n))), sa=z, ss=z.copy(),
                inflow=inflow, lmax=lmax, tol=tol)


def riemann_2d(n: int = 64, cfl: float = 2.0, lmax: int = 3, tol: float = 1e-10,
               sigma: float = 0.0) -> dict:
    """Section 5.2 Riemann problem in nondimensional form: [0,1]^2, four quadrants
    with F = (1 - 1e-8) c E F_hat, F_hat = (1,0) bottom-left, (0,-1) bottom-right,
    (0,1) top-left, (-1,0) top-right; uniform E = 1; periodic."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(x, x)
    fx = np.where((X < 0.5) & (Y < 0.5), 1.0, 0.0) + np.where((X >= 0.5) & (Y >= 0.5), -1.0, 0.0)
    fy = np.where((X >= 0.5) & (Y < 0.5), -1.0, 0.0) + np.where((X < 0.5) & (Y >= 0.5), 1.0, 0.0)
    k = 1.0 - 1e-8
    s = _state(n, n, np.ones((n, n)), k * fx, k * fy)
    return dict(desc=_desc(2, n, n, 1.0, 1.0, ["periodic"] * 4), dt=cfl * h, state=s,
                sa=np.full((n, n), sigma), ss=np.full((n, n), sigma), inflow=None, lmax=lmax,
                tol=tol)


def random_admissible_2d(nx: int, ny: int, seed: int, fmax: float = 0.999, cfl: float = 10.0,
                         bc=("periodic",) * 4, lmax: int = 2, tol: float = 1e-10,
                         dim: int = 2) -> dict:
    """Random admissible states: E log-uniform in [1e-2, 1e2], reduced flux f
    uniform in [0, fmax] with a uniform direction, T log-uniform in [0.5, 2],
    lognormal opacities.  A stress input for single kernels."""
    if dim == 1:
        ny = 1
    n = nx * ny
    E = 10.0 ** (4.0 * uniform(seed * 7 + 1, n) - 2.0)
    f = fmax * uniform(seed * 7 + 2, n)
    th = 2 * np.pi * uniform(seed * 7 + 3, n) if dim == 2 else np.where(
        uniform(seed * 7 + 3, n) < 0.5, 0.0, np.pi)
    T = 2.0 ** (2.0 * uniform(seed * 7 + 4, n) - 1.0)
    Fx, Fy = f * E * np.cos(th), f * E * np.sin(th)
    if dim == 1:
        Fy = np.zeros(n)
    s = np.stack([E, Fx, Fy, T]).reshape(4, ny, nx)
    h = 1.0 / nx
    sa = lognormal_opacity(nx, ny, seed * 7 + 5)
    ss = lognormal_opacity(nx, ny, seed * 7 + 6)
    inflow = None
    if "inflow" in bc:
        L = max(nx, ny)
        inflow = np.zeros((4, 3, L))
        inflow[:, 0, :] = 1.0
        inflow[:, 1, :] = 0.5
    return dict(desc=_desc(dim, nx, ny, 1.0, ny * h if dim == 2 else 1.0, list(bc)), dt=cfl * h,
                state=s, sa=sa, ss=ss, inflow=inflow, lmax=lmax, tol=tol)


def batched_instances(count: int = 512, seed: int = 5,
                      sizes=(64, 96, 128, 192, 256, 512, 1024), cfl: float = 100.0,
                      lmax: int = 5, tol: float = 1e-8) -> list:
    """Independent 2D instances: size drawn uniformly from `sizes` (square),
    per-instance lognormal opacities, E = 1 + A exp(-|x - x0|^2 / w) with
    A ~ U[1, 100], x0 ~ U[0.25, 0.75]^2, w ~ U[0.002, 0.02]; T = 1, F = 0,
    reflecting walls."""
    u = uniform(seed, 6 * count).reshape(count, 6)
    out = []
    for k in range(count):
        n = int(sizes[min(int(u[k, 0] * len(sizes)), len(sizes) - 1)])
        A = 1.0 + 99.0 * u[k, 1]
        x0, y0 = 0.25 + 0.5 * u[k, 2], 0.25 + 0.5 * u[k, 3]
        w = 0.002 + 0.018 * u[k, 4]
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        X, Y = np.meshgrid(x, x)
        E = 1.0 + A * np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / w)
        out.append(dict(desc=_desc(2, n, n, 1.0, 1.0, ["reflect"] * 4), dt=cfl * h,
                        state=_state(n, n, E), sa=lognormal_opacity(n, n, 1000 + 2 * k),
                        ss=lognormal_opacity(n, n, 1001 + 2 * k), inflow=None, lmax=lmax,
                        tol=tol))
    return out


def crop(case: dict, n: int, j0: int = 0, i0: int = 0) -> dict:
    """The n x n window of a 2D case starting at row j0, column i0 (same
    generator, smaller grid, same cell size and time step; the walls and the
    inflow profiles of the window's edges are the case's)."""
    c = dict(case)
    d = dict(case["desc"])
    h = d["lx"] / d["nx"]
    d.update(nx=n, ny=n, lx=n * h, ly=n * h)
    c["desc"] = d
    c["state"] = np.ascontiguousarray(case["state"][:, j0:j0 + n, i0:i0 + n])
    c["sa"] = np.ascontiguousarray(case["sa"][j0:j0 + n, i0:i0 + n])
    c["ss"] = np.ascontiguousarray(case["ss"][j0:j0 + n, i0:i0 + n])
    if case.get("inflow") is not None:
        # west/east walls are indexed by row, south/north walls by column
        fin = case["inflow"]
        inflow = np.zeros((4, 3, n))
        inflow[0:2] = fin[0:2, :, j0:j0 + n]
        inflow[2:4] = fin[2:4, :, i0:i0 + n]
        c["inflow"] = inflow
    return c


def beam_channel_crop(n: int = 1024, full: int = 4096, lmax: int = 8, tol: float = 1e-8) -> dict:
    """The n x n window of the full x full beam-in-a-channel case that holds the
    beam: on the west wall, centred on the channel (rows full/2 - n/2 ...)."""
    return dict(crop(beam_channel_2d(full, lmax=lmax, tol=tol), n, j0=(full - n) // 2, i0=0),
                lmax=lmax)


def bump_case(dim: int, n: int, seed: int, cfl: float, lmax: int, tol: float) -> dict:
    """One instance: E = 1e-2 + A exp(-|x - x0|^2 / w) with A ~ U[1, 100],
    x0 ~ U[0.25, 0.75]^d, w ~ U[0.002, 0.02]; T = 1, F = 0; lognormal sigma_a,
    sigma_s; 1D periodic, 2D reflecting walls; dt = cfl * h / c."""
    u = uniform(seed, 4)
    A, w = 1.0 + 99.0 * u[0], 0.002 + 0.018 * u[3]
    x0, y0 = 0.25 + 0.5 * u[1], 0.25 + 0.5 * u[2]
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    if dim == 1:
        E = 1e-2 + A * np.exp(-(x - x0) ** 2 / w)
        return dict(desc=_desc(1, n, 1, 1.0, 1.0, ["periodic"] * 4), dt=cfl * h,
                    state=_state(n, 1, E[None, :]), sa=lognormal_opacity(n, 1, 2 * seed + 1),
                    ss=lognormal_opacity(n, 1, 2 * seed + 2), inflow=None, lmax=lmax, tol=tol)
    X, Y = np.meshgrid(x, x)
    E = 1e-2 + A * np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / w)
    return dict(desc=_desc(2, n, n, 1.0, 1.0, ["reflect"] * 4), dt=cfl * h, state=_state(n, n, E),
                sa=lognormal_opacity(n, n, 2 * seed + 1), ss=lognormal_opacity(n, n, 2 * seed + 2),
                inflow=None, lmax=lmax, tol=tol)


def serving_stream(count: int = 64, seed: int = 11, rate_hz: float = 20.0,
                   sizes_1d=(256, 512, 1024, 2048, 4096, 8192, 16384, 32768, 65536),
                   sizes_2d=(128, 256, 512, 1024, 2048), steps=(10, 100),
                   cfl_1d: float = 50.0, cfl_2d: float = 100.0, lmax: int = 5,
                   tol: float = 1e-8) -> list:
    """Requests of a Poisson arrival stream of simulations: exponential arrival
    gaps of mean 1 / rate_hz (inverse transform of uniforms), 1D or 2D with
    probability 1/2, the size uniform over the given set, the number of steps
    uniform over [steps[0], steps[1]]; each request is a bump_case.  Returns
    dicts {case, nsteps, arrival_s} in arrival order."""
    u = uniform(seed, 4 * count).reshape(count, 4)
    t = 0.0
    out = []
    for k in range(count):
        t += -np.log1p(-u[k, 0]) / rate_hz
        if u[k, 1] < 0.5:
            n = int(sizes_1d[min(int(u[k, 2] * len(sizes_1d)), len(sizes_1d) - 1)])
            case = bump_case(1, n, 7000 + k, cfl_1d, lmax, tol)
        else:
            n = int(sizes_2d[min(int(u[k, 2] * len(sizes_2d)), len(sizes_2d) - 1)])
            case = bump_case(2, n, 7000 + k, cfl_2d, lmax, tol)
        nsteps = steps[0] + min(int(u[k, 3] * (steps[1] - steps[0] + 1)), steps[1] - steps[0])
        out.append(dict(case=case, nsteps=int(nsteps), arrival_s=t))
    return out
