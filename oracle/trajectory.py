"""One time step of a monitored Gaussian trajectory (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

State.  App. A writes the Slater determinant as
|psi> = prod_k (sum_j U_jk c_j^dag) |vac>, U an L x N matrix with U^dag U = 1.
The correlation matrix D_ij = <c_i^dag c_j> of Sec. II equals conj(U U^dag);
this module works with C = U U^dag, which has the same eigenvalues, the same
|C_ij| and obeys the same update formulas.

A step t -> t + dt (fixed dt) is

1. unitary propagation U <- P U with P = exp(-i H~ dt)  (App. A);
2. the measurement:
   * projective protocol (App. A): each site j is measured with probability
     1 - exp(-gamma dt), the sites in ascending order; the Born probability is
     p_j = C_jj of the current state and the outcome is 1 when the uniform
     draw u_j < p_j.  A click projects with n_j (Eq. (A1)), a no-click with
     1 - n_j (Eq. (A2), with the sign of its correction term read as '+',
     the form that conserves particle number).  Both are applied to U as the
     rank-1 updates derived in ``project_site``;
   * homodyne / QSD protocol (Eq. (A4)): U <- exp(dW + (2<n> - 1) gamma dt) U
     with dW_i = sqrt(gamma dt) xi_i, xi_i ~ N(0,1), and <n_i> = sum_k |U_ik|^2
     of the propagated state;
   * the same protocol integrated as App. A does it (``HOMODYNE_RK4``): steps 1
     and 2 together as one Runge-Kutta step of Eq. (QSD_evo) (``step_rk4``);
3. re-orthonormalisation U <- Q of U = QR (App. A), every step for the
   homodyne protocol and every ``reorth_interval`` steps for the projective one
   (whose rank-1 updates keep U^dag U = 1 up to rounding).
"""
from dataclasses import dataclass

import numpy as np

from . import lattice, philox

PROJECTIVE = 0
HOMODYNE = 1
HOMODYNE_RK4 = 2       # App. A's own integrator for Eq. (QSD_evo), see ``step_rk4``
PROJECTIVE_POISSON = 3 # App. A's own continuous-time projective protocol, see ``run_poisson``


@dataclass
class Params:
    Lx: int
    Ly: int = 1
    J: float = 1.0
    dt: float = 0.05
    gamma: float = 0.5
    protocol: int = PROJECTIVE
    reorth_interval: int = 1
    seed: int = 0
    traj_id: int = 0

    @property
    def L(self):
        return self.Lx * self.Ly

    @property
    def N(self):
        return len(lattice.occupied_sites(self.Lx, self.Ly))


def orthonormalize(U):
    """Q factor of the Householder QR U = QR (App. A)."""
    Q, _ = np.linalg.qr(U)
    return Q


def occupations(U):
    """<n_i> = sum_k U_ik conj(U_ik) (App. A, below Eq. (A4))."""
    return np.real(np.sum(U * np.conj(U), axis=1))


def homodyne_weight(U, xi, gamma, dt):
    """U <- exp(dW + (2<n> - 1) gamma dt) U, dW_i = sqrt(gamma dt) xi_i (Eq. (A4))."""
    n = occupations(U)
    m = np.sqrt(gamma * dt) * xi + (2.0 * n - 1.0) * gamma * dt
    return np.exp(m)[:, None] * U


def project_site(U, j, outcome):
    """Apply n_j (outcome 1) or 1 - n_j (outcome 0) to the Slater determinant.

    With x = U_{j,:}, p = |x|^2 = C_jj and the unit orbital-space vector
    xh = x^dag / sqrt(p), the orbitals orthogonal to xh have no weight on
    site j, and U xh = v = C_{:,j} / sqrt(p).  n_j replaces v by e_j;
    1 - n_j replaces v by (v - sqrt(p) e_j) / sqrt(1 - p).  Either way only the
    xh direction changes, so U <- U + (v_new - v) xh^dag keeps U^dag U = 1.
    On C = U U^dag this is Eq. (A1) for a click and Eq. (A2) (with '+') for
    no click.
    """
    x = U[j, :].copy()
    p = float(np.real(np.vdot(x, x)))
    p = min(max(p, 0.0), 1.0)
    sp = np.sqrt(p)
    v = (U @ np.conj(x)) / sp
    ej = np.zeros(U.shape[0], dtype=U.dtype)
    ej[j] = 1.0
    if outcome == 1:
        v_new = ej
    else:
        v_new = (v - sp * ej) / np.sqrt(1.0 - p)
    return U + np.outer(v_new - v, x) / sp


def projective_measurements(U, p_meas, u_sel, u_out, forced=None):
    """Measure the selected sites of one step in ascending order.

    ``forced`` optionally maps site -> outcome to replay a given sequence.
    Returns the new U and the event list [(site, u, p, outcome)].
    """
    events = []
    for j in np.nonzero(u_sel < p_meas)[0]:
        j = int(j)
        x = U[j, :]
        p = min(max(float(np.real(np.vdot(x, x))), 0.0), 1.0)
        outcome = 1 if u_out[j] < p else 0
        if forced is not None and j in forced:
            outcome = forced[j]
        events.append((j, float(u_out[j]), p, outcome))
        if p < 1e-300:
            continue          # no weight on site j: a no-click leaves the state unchanged
        U = project_site(U, j, outcome)
    return U, events


def step_rk4(U, H, xi, gamma, dt):
    """One step of Eq. (QSD_evo) by the classical fourth-order Runge-Kutta method (App. A).

    Over the step the noise dW_i = sqrt(gamma dt) xi_i and <n_i>_t (of the state at the
    start of the step) are held fixed, so dU/dt = A U with the constant matrix
    A dt = -i dt H~ + diag(m), m_i = dW_i + (2 <n_i>_t - 1) gamma dt.  The four RK4 stages
    k1 = A U, k2 = A (U + dt k1 / 2), k3 = A (U + dt k2 / 2), k4 = A (U + dt k3) give
    U + dt (k1 + 2 k2 + 2 k3 + k4) / 6.  The caller re-orthonormalises.
    """
    n = occupations(U)
    m = np.sqrt(gamma * dt) * xi + (2.0 * n - 1.0) * gamma * dt
    A = -1j * H + np.diag(m / dt)
    k1 = A @ U
    k2 = A @ (U + 0.5 * dt * k1)
    k3 = A @ (U + 0.5 * dt * k2)
    k4 = A @ (U + dt * k3)
    return U + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def step(U, P, prm, step_index, forced=None, H=None):
    """Advance U from t = step_index*dt to t + dt.  Returns (U, events).

    P is the propagator of the split step; H (the hopping matrix) is used by the
    Runge-Kutta protocol instead."""
    L = U.shape[0]
    events = []
    if prm.protocol == HOMODYNE_RK4:
        if H is None:
            H = lattice.hopping_matrix(prm.Lx, prm.Ly, prm.J)
        xi = philox.noise_normals(prm.seed, prm.traj_id, step_index, L)
        return orthonormalize(step_rk4(U, H, xi, prm.gamma, prm.dt)), events
    U = P @ U
    if prm.protocol == HOMODYNE:
        xi = philox.noise_normals(prm.seed, prm.traj_id, step_index, L)
        U = orthonormalize(homodyne_weight(U, xi, prm.gamma, prm.dt))
    else:
        u_sel, u_out = philox.measure_draws(prm.seed, prm.traj_id, step_index, L)
        p_meas = 1.0 - np.exp(-prm.gamma * prm.dt)
        U, events = projective_measurements(U, p_meas, u_sel, u_out, forced)
        if (step_index + 1) % prm.reorth_interval == 0:
            U = orthonormalize(U)
    return U, events


def run_poisson(prm, nsteps, U=None, forced=None):
    """The projective protocol as App. A runs it, in continuous time.

    Measurement events come at the times of a Poisson process of total rate gamma N
    (N = L/2 particles; the waiting time of event e is -ln(1 - u_wait) / (gamma N), the
    form of tau = ln(eta) / (gamma N) with the sign that makes it positive); at each
    event one site j, uniform over the L sites, is measured with the Born weight
    p = C_jj and the outcome u < p, by the same rank-1 updates as the fixed-dt
    protocol; between events the state evolves by exp(-i H~ tau) (here ``expm``).  The
    events are a fixed sequence per trajectory (``philox.poisson_event``), their times
    the running sum of the waiting times; step s covers (s dt, (s+1) dt] and ends with
    the propagation to (s+1) dt.  QR every ``reorth_interval`` steps.  ``forced``
    optionally maps event index -> outcome to replay a given sequence.
    Returns dict(U, events=[(step, site, u, p, outcome)]).
    """
    import scipy.linalg
    L = prm.L
    N = prm.N
    H = lattice.hopping_matrix(prm.Lx, prm.Ly, prm.J)
    if U is None:
        U = lattice.initial_orbitals(prm.Lx, prm.Ly)
    rate = prm.gamma * N
    e = 0
    t_next = np.inf
    if rate > 0:
        t_next = -np.log1p(-philox.poisson_event(prm.seed, prm.traj_id, 0, L)[0]) / rate
    t = 0.0
    events = []
    for s in range(nsteps):
        t1 = (s + 1) * prm.dt
        while t_next <= t1:
            U = scipy.linalg.expm(-1j * (t_next - t) * H) @ U
            t = t_next
            _, j, u = philox.poisson_event(prm.seed, prm.traj_id, e, L)
            x = U[j, :]
            p = min(max(float(np.real(np.vdot(x, x))), 0.0), 1.0)
            outcome = 1 if u < p else 0
            if forced is not None and e in forced:
                outcome = forced[e]
            events.append((s, j, u, p, outcome))
            if p >= 1e-300:
                U = project_site(U, j, outcome)
            e += 1
            t_next = t_next + (-np.log1p(-philox.poisson_event(prm.seed, prm.traj_id, e, L)[0]) / rate)
        U = scipy.linalg.expm(-1j * (t1 - t) * H) @ U
        t = t1
        if (s + 1) % prm.reorth_interval == 0:
            U = orthonormalize(U)
    return {"U": U, "events": events}


def run(prm, nsteps, U=None, P=None, start_step=0, ee_every=0, ee_sites=None, forced=None):
    """Run ``nsteps`` steps.  Returns dict(U, events, ee=[(steps_done, S)]).

    ``forced`` optionally maps step index -> {site: outcome} (the continuous-time
    protocol: event index -> outcome).
    """
    from . import observables
    if prm.protocol == PROJECTIVE_POISSON:
        if start_step or ee_every:
            raise ValueError("run_poisson: whole trajectories from t = 0 only")
        out = run_poisson(prm, nsteps, U, forced)
        out["ee"] = []
        return out
    H = None
    if prm.protocol == HOMODYNE_RK4:
        H = lattice.hopping_matrix(prm.Lx, prm.Ly, prm.J)
    elif P is None:
        P = lattice.propagator(prm.Lx, prm.Ly, prm.J, prm.dt)
    if U is None:
        U = lattice.initial_orbitals(prm.Lx, prm.Ly)
    events, ee = [], []
    for s in range(start_step, start_step + nsteps):
        U, ev = step(U, P, prm, s, None if forced is None else forced.get(s), H=H)
        events.extend((s,) + e for e in ev)
        done = s + 1
        if ee_every and ee_sites is not None and done % ee_every == 0:
            ee.append((done, observables.entanglement_entropy(U, ee_sites)))
    return {"U": U, "events": events, "ee": ee}
