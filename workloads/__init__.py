"""Seeded synthetic inputs for the FMM vortex-particle workloads.

Input generation only: this module holds none of the method's arithmetic and
is shared by the tests, the benchmark and the oracle checks.  Every generator
is seeded (numpy Philox, seed = 20111106 + workload id unless given) and
returns float32 positions/strengths as the GPU receives them.

Workloads (all sizes as used by the benchmark and the parity tests):
  jittered_lattice  N = n^3 blobs on a jittered lattice in the unit cube
                    (spacing h = 1/n, points (i+1/2)h, jitter U(+-0.25h)),
                    gamma ~ N(0,1)^3 drawn in FP64 then rounded, sigma = 1.5h,
                    free space.  n = 16 is the 4096-blob accuracy case.
  taylor_green      N = n^3 blobs on the lattice (i+1/2)h of the periodic cube
                    [0, 2 pi)^3, h = 2 pi/n, gamma = omega_TG(x) h^3 with
                    u_TG = (sin x cos y cos z, -cos x sin y cos z, 0),
                    sigma = 1.2h.  n = 128 is the 2,097,152-blob benchmark.
  random_spectrum   Lattice in [0, 2 pi)^3 with vorticity of a random-phase
                    solenoidal field, E(k) ~ k^4 exp(-2 (k/k0)^2), k0 = 4,
                    u_rms = 1, gamma = omega h^3, sigma = 1.2h.  Also returns
                    the Fourier modes so the velocity can be evaluated exactly.
  uniform_ball / plummer   clustered free-space inputs with Gaussian strengths.
"""
import math

import numpy as np

BASE_SEED = 20111106


def rng(seed):
    return np.random.Generator(np.random.Philox(seed))


def jittered_lattice(n=16, seed=BASE_SEED + 1):
    g = rng(seed)
    h = 1.0 / n
    i = (np.arange(n) + 0.5) * h
    X, Y, Z = np.meshgrid(i, i, i, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    pos = pos + g.uniform(-0.25 * h, 0.25 * h, size=pos.shape)
    gamma = g.standard_normal(size=pos.shape)
    return dict(pos=pos.astype(np.float32), gamma=gamma.astype(np.float32),
                sigma=np.float32(1.5 * h), periodic=False, p=6, theta=0.5, ncrit=32,
                name="jittered-lattice-%d^3" % n)


def _tg_vorticity(x):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    return np.stack([-np.cos(X) * np.sin(Y) * np.sin(Z),
                     -np.sin(X) * np.cos(Y) * np.sin(Z),
                     2.0 * np.sin(X) * np.sin(Y) * np.cos(Z)], 1)


def taylor_green(n=128):
    L = 2.0 * math.pi
    h = L / n
    i = (np.arange(n) + 0.5) * h
    X, Y, Z = np.meshgrid(i, i, i, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    pos32 = pos.astype(np.float32)
    gamma = _tg_vorticity(pos32.astype(np.float64)) * h ** 3
    return dict(pos=pos32, gamma=gamma.astype(np.float32), sigma=np.float32(1.2 * h),
                periodic=True, box_min=np.zeros(3), box_len=L, p=10, theta=0.4, ncrit=64,
                images=3, name="taylor-green-%d^3" % n)


def random_spectrum(n=64, k0=4.0, seed=BASE_SEED + 3, kmax=None):
    """Random-phase solenoidal field on an n^3 lattice; returns its Fourier modes too.

    Modes k (integer wave vectors, one of each +-k pair) with |k| <= kmax carry
    u_hat(k) = P_perp(k) xi(k) sqrt(E(k) / (4 pi k^2)), xi complex Gaussian,
    E(k) = k^4 exp(-2 (k/k0)^2), scaled to u_rms = 1; the vorticity at the
    lattice points (i+1/2)h is the real part of 2 sum_k i k x u_hat e^{i k.x},
    evaluated by an inverse FFT (the half-cell offset as a phase factor).
    """
    g = rng(seed)
    L = 2.0 * math.pi
    h = L / n
    if kmax is None:
        kmax = min(n // 2 - 1, int(5 * k0))
    r = np.arange(-kmax, kmax + 1)
    KX, KY, KZ = np.meshgrid(r, r, r, indexing="ij")
    k = np.stack([KX.ravel(), KY.ravel(), KZ.ravel()], 1).astype(np.float64)
    kk = np.sqrt((k * k).sum(1))
    keep = (kk > 0) & (kk <= kmax)
    first = (k[:, 0] > 0) | ((k[:, 0] == 0) & (k[:, 1] > 0)) | ((k[:, 0] == 0) & (k[:, 1] == 0) & (k[:, 2] > 0))
    keep &= first
    k = k[keep]
    kk = kk[keep]
    E = kk ** 4 * np.exp(-2.0 * (kk / k0) ** 2)
    xi = g.standard_normal((k.shape[0], 3)) + 1j * g.standard_normal((k.shape[0], 3))
    khat = k / kk[:, None]
    xi = xi - (xi * khat).sum(1)[:, None] * khat  # solenoidal projection
    uhat = xi * np.sqrt(E / (4.0 * math.pi * kk ** 2))[:, None]
    # u_rms over the lattice = sqrt(2 sum |u_hat|^2) for a sum over +-k pairs
    uhat /= math.sqrt(2.0 * (np.abs(uhat) ** 2).sum())
    what = 1j * np.cross(k, uhat)
    # grid spectrum: f(x_i) = sum_k [c(k) e^{i k h/2}] e^{i k . (i h)}, both k and -k
    ki = k.astype(np.int64)
    grid = np.zeros((3, n, n, n), np.complex128)
    ph = np.exp(0.5j * h * k.sum(1))
    for sgn, coef, pf in ((1, what, ph), (-1, np.conj(what), np.conj(ph))):
        idx = tuple((sgn * ki[:, a]) % n for a in range(3))
        for c in range(3):
            np.add.at(grid[c], idx, coef[:, c] * pf)
    w = np.stack([np.real(np.fft.ifftn(grid[c])) * n ** 3 for c in range(3)], -1).reshape(-1, 3)
    i1 = (np.arange(n) + 0.5) * h
    X, Y, Z = np.meshgrid(i1, i1, i1, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    gamma = w * h ** 3
    return dict(pos=pos.astype(np.float32), gamma=gamma.astype(np.float32), sigma=np.float32(1.2 * h),
                periodic=True, box_min=np.zeros(3), box_len=L, p=10, theta=0.4, ncrit=64,
                images=3, modes=k, uhat=uhat, name="random-spectrum-%d^3" % n)


def uniform_ball(n, seed=BASE_SEED + 4):
    g = rng(seed)
    v = g.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    r = g.random(n) ** (1.0 / 3.0)
    pos = v * r[:, None]
    gamma = g.standard_normal((n, 3))
    sigma = 1.5 * (4.0 / 3.0 * math.pi / n) ** (1.0 / 3.0)
    return dict(pos=pos.astype(np.float32), gamma=gamma.astype(np.float32),
                sigma=np.float32(sigma), periodic=False, name="ball-%d" % n)


def plummer_sigma(n, a=0.1):
    """Core width for a Plummer cloud of n blobs: 1.5 x the mean spacing inside
    the half-mass radius r_h = a / sqrt(2^(2/3) - 1) (n/2 blobs there), so the
    near field of the dense core stays a few thousand neighbours as for a
    uniform cloud (a width from the spacing of the whole unit ball would put
    most of the core inside 5 sigma of every core blob)."""
    rh = a / math.sqrt(2.0 ** (2.0 / 3.0) - 1.0)
    return 1.5 * (4.0 / 3.0 * math.pi * rh ** 3 / max(n / 2.0, 1.0)) ** (1.0 / 3.0)


def plummer(n, a=0.1, seed=BASE_SEED + 5, sigma_rule="ball"):
    g = rng(seed)
    X = g.random(2 * n + 16)
    X = X[X < 0.999][:n]
    while X.shape[0] < n:
        extra = g.random(n)
        X = np.concatenate([X, extra[extra < 0.999]])[:n]
    r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    v = g.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    pos = v * r[:, None]
    gamma = g.standard_normal((n, 3))
    if sigma_rule == "halfmass":
        sigma = plummer_sigma(n, a)
    else:
        sigma = 1.5 * (4.0 / 3.0 * math.pi / n) ** (1.0 / 3.0)
    return dict(pos=pos.astype(np.float32), gamma=gamma.astype(np.float32),
                sigma=np.float32(sigma), periodic=False, name="plummer-%d" % n)


def batch_specs(nprob=512, nmin=1e3, nmax=1e6, orders=(4, 8, 12), seed=BASE_SEED + 4):
    """Independent free-space problems for a batched evaluation: N log-uniform
    in [nmin, nmax], positions uniform in the unit ball or Plummer-clustered
    (a = 0.1) with equal odds, Gaussian strengths, sigma = 1.5 (V_ball/N)^(1/3)
    for the ball and plummer_sigma(N) for the clusters, expansion order drawn
    from `orders`.  Returns specs; make_problem builds one."""
    g = rng(seed)
    N = np.exp(g.uniform(math.log(nmin), math.log(nmax), nprob)).astype(np.int64)
    kind = g.integers(0, 2, nprob)
    p = g.choice(np.asarray(orders), nprob)
    seeds = g.integers(0, 2 ** 31, nprob)
    return [dict(n=int(N[k]), kind=("ball", "plummer")[int(kind[k])], p=int(p[k]), seed=int(seeds[k]),
                 periodic=False) for k in range(nprob)]


def request_specs(rate=200.0, horizon_s=60.0, nmin=1e4, nmax=4e6, orders=(4, 8, 12), periodic_frac=0.3,
                  seed=BASE_SEED + 5):
    """A Poisson request stream: arrival times with mean rate `rate` per second
    over `horizon_s`, N log-uniform in [nmin, nmax], order from `orders`;
    `periodic_frac` of the requests are random-spectrum blobs on a ceil(N^(1/3))^3
    lattice in the periodic cube [0, 2 pi)^3, the rest Plummer-clustered free-space
    problems.  Returns specs sorted by arrival time."""
    g = rng(seed)
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate)
        if t >= horizon_s:
            break
        n = int(math.exp(g.uniform(math.log(nmin), math.log(nmax))))
        per = bool(g.random() < periodic_frac)
        if per:
            m = int(math.ceil(n ** (1.0 / 3.0)))
            n = m ** 3
        out.append(dict(t=t, n=n, kind="spectrum" if per else "plummer", p=int(g.choice(np.asarray(orders))),
                        seed=int(g.integers(0, 2 ** 31)), periodic=per))
    return out


def make_problem(spec):
    """Particles of one batch_specs / request_specs entry."""
    if spec["kind"] == "ball":
        return uniform_ball(spec["n"], seed=spec["seed"])
    if spec["kind"] == "plummer":
        return plummer(spec["n"], seed=spec["seed"], sigma_rule="halfmass")
    m = int(round(spec["n"] ** (1.0 / 3.0)))
    return random_spectrum(m, seed=spec["seed"])


def random_cloud(n, seed=BASE_SEED + 6, box=1.0, zero_net=False):
    g = rng(seed)
    pos = g.random((n, 3)) * box
    gamma = g.standard_normal((n, 3))
    if zero_net and n > 0:
        gamma -= gamma.mean(0)
    return dict(pos=pos.astype(np.float32), gamma=gamma.astype(np.float32))
