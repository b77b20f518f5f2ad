"""Seeded workload generators (numpy.random.default_rng, float64).

Every generator returns plain numpy arrays.  A system is a dict with keys
  A (n,n), B (n,m)            linear dynamics  xdot = A x + B u      (§II.B, Eq. 8)
  ctrl_kind  0 = ball, 1 = box
  radius     ball radius rho   (ball control set {|u|_2 <= rho})
  half_widths (m,)             box half widths b (box control set {|u_j| <= b_j})
  W (n,n)                      SPD shape of the target {x : x^T W^-1 x <= 1}  (Eq. 34)
The shapes and value distributions follow the five benchmark workloads; the
paper's own examples (§VI) are the double integrator and stacked copies of it.
"""
import numpy as np

BALL, BOX = 0, 1
LEFT_RIEMANN, TRAPEZOID, SIMPSON = 0, 1, 2


def double_integrator(radius_target=0.1, u_max=1.0):
    """Double integrator of §VI.A: position/velocity, scalar control |u| <= u_max,
    circular target of the given radius (W = r^2 I)."""
    return dict(A=np.array([[0.0, 1.0], [0.0, 0.0]]), B=np.array([[0.0], [1.0]]),
                ctrl_kind=BOX, radius=1.0, half_widths=np.array([u_max]),
                W=(radius_target ** 2) * np.eye(2))


def single_integrator(n, ctrl_kind=BALL, radius=1.0, radius_target=0.5):
    """xdot = u in R^n (A = 0, B = I): the setting of the basic Hopf formula (Eq. 6)."""
    return dict(A=np.zeros((n, n)), B=np.eye(n), ctrl_kind=ctrl_kind, radius=radius,
                half_widths=np.full(n, radius), W=(radius_target ** 2) * np.eye(n))


def random_system(seed, n=10, m=2):
    """Random controllable-looking system: A_ij ~ N(0, 1/n) - 0.5 delta_ij,
    B_ij ~ N(0, 1); unit 2-norm ball control; ellipsoid target x^T Q x <= 1 with
    Q = diag(q), q_j ~ U[1, 4] (so W = diag(1/q)).  Draw order: A, B, q."""
    rng = np.random.default_rng(seed)
    A = rng.normal(0.0, np.sqrt(1.0 / n), (n, n)) - 0.5 * np.eye(n)
    B = rng.normal(0.0, 1.0, (n, m))
    q = rng.uniform(1.0, 4.0, n)
    return dict(A=A, B=B, ctrl_kind=BALL, radius=1.0, half_widths=np.ones(m),
                W=np.diag(1.0 / q))


def spring_chain(masses=100, k=1.0, damping=0.1, actuators=10, u_max=1.0, radius_target=0.5):
    """Chain of unit masses between two fixed walls; springs of stiffness k between
    neighbours and to each wall; viscous damping on every mass.  State [q; v]
    (n = 2*masses); actuators on masses 10j+5 (0-based), box |u_i| <= u_max;
    ball target of the given radius."""
    nm = masses
    Ks = np.zeros((nm, nm))
    for i in range(nm):
        Ks[i, i] = 2.0 * k
        if i > 0:
            Ks[i, i - 1] = -k
        if i + 1 < nm:
            Ks[i, i + 1] = -k
    A = np.zeros((2 * nm, 2 * nm))
    A[:nm, nm:] = np.eye(nm)
    A[nm:, :nm] = -Ks
    A[nm:, nm:] = -damping * np.eye(nm)
    E = np.zeros((nm, actuators))
    for j in range(actuators):
        E[(nm // actuators) * j + (nm // actuators) // 2, j] = 1.0
    B = np.zeros((2 * nm, actuators))
    B[nm:, :] = E
    return dict(A=A, B=B, ctrl_kind=BOX, radius=1.0, half_widths=np.full(actuators, u_max),
                W=(radius_target ** 2) * np.eye(2 * nm))


def normal_points(seed, P, n, std):
    """P query points x ~ N(0, std^2 I)."""
    return np.random.default_rng(seed).normal(0.0, std, (P, n))


def uniform_points(seed, P, n, lo, hi):
    """P query points uniform in the box [lo, hi]^n."""
    return np.random.default_rng(seed).uniform(lo, hi, (P, n))


def grid_points(k, lo, hi):
    """k x k grid on [lo, hi]^2 (the 50 x 50 grid of the double-integrator example)."""
    g = np.linspace(lo, hi, k)
    X, Y = np.meshgrid(g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


# ---------------------------------------------------------------- named workloads
def workload_di(P=64):
    """Double integrator, box |u| <= 1, ball target r = 0.1, P points uniform in
    [-2, 2]^2, trapezoid rule with 128 nodes, FP64, gap 1e-8, bisection on [0, 10]."""
    sysd = double_integrator(0.1)
    return dict(name="double_integrator_fp64", system=sysd,
                x=uniform_points(0, P, 2, -2.0, 2.0), rule=TRAPEZOID, N=128,
                tol_gap=1e-8, t_max=10.0, tau=2.0)


def workload_random10(P=65536, seed_sys=1, seed_pts=2):
    """One random n=10, m=2 system, unit ball control, ellipsoid target;
    P points x ~ N(0, 4 I); fixed horizon t = 2; left Riemann with 256 nodes."""
    sysd = random_system(seed_sys, 10, 2)
    return dict(name="random_n10_m2_fp32", system=sysd, x=normal_points(seed_pts, P, 10, 2.0),
                t=2.0, rule=LEFT_RIEMANN, N=256, tol_gap=1e-5, tau=0.15)


def workload_ragged(systems=64, seed_layout=99):
    """64 random systems as above with n uniform in {4..128}, m = ceil(n/8), and
    1000..4000 points each (x ~ N(0, 4 I)); fixed horizon t = 2; 256 nodes."""
    rng = np.random.default_rng(seed_layout)
    ns = rng.integers(4, 129, systems)
    Ps = rng.integers(1000, 4001, systems)
    out = []
    for s in range(systems):
        n = int(ns[s]); m = int(np.ceil(n / 8))
        out.append(dict(system=random_system(100 + s, n, m),
                        x=normal_points(200 + s, int(Ps[s]), n, 2.0)))
    return dict(name="ragged_64_systems", items=out, t=2.0, rule=LEFT_RIEMANN, N=256,
                tol_gap=1e-5)


def workload_chain(P=4096):
    """100-mass spring chain (n=200, m=10, box control), ball target r = 0.5;
    P points x ~ N(0, I); 512 nodes; time-to-reach and 1000-sample trajectories."""
    return dict(name="spring_chain_n200", system=spring_chain(), x=normal_points(3, P, 200, 1.0),
                rule=LEFT_RIEMANN, N=512, tol_gap=1e-5, samples=1000)


def stacked_copies(base, k, block_scale):
    """k copies of a base system driven by one shared control (§VI.B): state
    (chi_1, ..., chi_k), A~ = blockdiag(A, ..., A), B~ = (B; ...; B); target
    weight W = blockdiag(block_scale[j] I) (Omega = {x^T W^-1 x <= 1})."""
    A, B = base["A"], base["B"]
    nb = A.shape[0]
    out = dict(base)
    out["A"] = np.kron(np.eye(k), A)
    out["B"] = np.kron(np.ones((k, 1)), B)
    out["W"] = np.kron(np.diag(np.asarray(block_scale, dtype=np.float64)), np.eye(nb))
    out["base"] = dict(base)
    out["W_blocks"] = np.asarray(block_scale, dtype=np.float64)[:, None, None] * np.eye(nb)[None]
    return out


def unscented_samples(mu, std, kappa=1.0):
    """2 d + 1 sigma points of N(mu, std^2 I) in d dimensions and their mean
    weights (scaled unscented transform with alpha = 1, beta unused, kappa):
    lambda = kappa, chi_0 = mu, chi_{+-j} = mu +- sqrt(d + lambda) std e_j,
    w_0 = lambda / (d + lambda), w_j = 1 / (2 (d + lambda))."""
    mu = np.asarray(mu, dtype=np.float64)
    d = mu.shape[-1]
    lam = kappa
    h = np.sqrt(d + lam) * std
    pts = [mu] + [mu + h * e for e in np.eye(d)] + [mu - h * e for e in np.eye(d)]
    w = np.array([lam / (d + lam)] + [1.0 / (2.0 * (d + lam))] * (2 * d))
    return np.stack(pts, axis=-2), w


def workload_unscented(P=64, ell=0.1, std=0.0667, seed=12):
    """§VI.B: the double integrator with an uncertain initial state N(mu, std^2 I)
    represented by its 5 sigma points, one shared control (n = 10, m = 1 box).
    Terminal cost sum_j w_j |chi_j|^2 - ell (the weighted mean square distance
    to the origin) = ell (x^T W^-1 x - 1) with W = ell blockdiag(I / w_j): same
    zero level set and time-to-reach as the paper's cost.  P query means
    mu ~ U[-1, 1]^2; left Riemann, N = 100, tau = 0.5 (the paper's value).
    The spread of the copies cannot be steered away, so phi(x, T) rises again
    for large T; time-to-reach brackets on [0, 4], below that rise."""
    mus = uniform_points(seed, P, 2, -1.0, 1.0)
    chis, wm = unscented_samples(mus, std)
    sysd = stacked_copies(double_integrator(0.1), len(wm), ell / wm)
    return dict(name="unscented_double_integrator_n10", system=sysd, x=chis.reshape(P, -1), mu=mus,
                weights=wm, ell=ell, rule=LEFT_RIEMANN, N=100, tau=0.5, tol_gap=1e-5, t_max=4.0)


def workload_dimension(d, P=64, ell=0.1, std=0.0667, seed=13):
    """§VI.C dimensional scaling: k = d / 2 double-integrator samples
    chi_j ~ N(mu, std^2 I) (iid, seeded) sharing one control (n = d, m = 1 box),
    terminal cost (1/k) sum_j |chi_j|^2 - ell, i.e. W = ell k I; P query means
    mu ~ U[-1, 1]^2; left Riemann, N = 100, tau = 0.5."""
    k = d // 2
    rng = np.random.default_rng(seed)
    mus = rng.uniform(-1.0, 1.0, (P, 2))
    chis = mus[:, None, :] + std * rng.normal(0.0, 1.0, (P, k, 2))
    sysd = stacked_copies(double_integrator(0.1), k, np.full(k, ell * k))
    return dict(name=f"dimension_scaling_d{d}", system=sysd, x=chis.reshape(P, -1), mu=mus, ell=ell,
                rule=LEFT_RIEMANN, N=100, tau=0.5, tol_gap=1e-5, t_max=10.0)


def mlp_init(seed, sizes):
    """He-style initial weights for an MLP with the given layer sizes.  Returns a list
    of (W (out,in), b (out,)) pairs in float64."""
    rng = np.random.default_rng(seed)
    layers = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        layers.append((rng.normal(0.0, np.sqrt(2.0 / fan_in), (fan_out, fan_in)),
                       np.zeros(fan_out)))
    return layers
