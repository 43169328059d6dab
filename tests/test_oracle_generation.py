"""Pins of the oracle's trajectory generation (Section IV-B) against closed forms and invariants.

Nothing here re-types the oracle's update rule: every expected value comes from a different route
(kinematics in closed form, the steady state of the linear bicycle model, convergence order, symmetry).
"""
import math

import numpy as np
import pytest

from paper_2005_06773_gb300 import scenarios as S

CAR = dict(length=4.5, width=1.8)


def car(x0=0.0, y0=0.0, psi0=0.0, v0=10.0, acc=(0.0,), steer=(0.0,), params=None):
    return S.Obj(S.VEHICLE, 4.5, 1.8, 0.0, x0, y0, psi0, v0, np.array(acc), np.array(steer),
                 S.DEFAULT_VEH_PARAMS if params is None else params)


def ped(x0=0.0, y0=0.0, psi0=0.0, v0=0.0, grid_a=(1.0,), grid_b=(0.0,), v_max=0.0, flags=0):
    return S.Obj(S.PEDESTRIAN, 0.0, 0.0, 0.4, x0, y0, psi0, v0, np.array(grid_a), np.array(grid_b),
                 v_max=v_max, flags=flags)


def gen(orc, objs, tau=0.1, n=30, k=5, model=S.MODEL_OT):
    return orc.generate(S.Scenario(objs, tau=tau, n_steps=n, substeps=k, model=model))


def times(tau, n):
    return (np.arange(n) + 1) * float(np.float32(tau))


@pytest.mark.parametrize("model", [S.MODEL_OT, S.MODEL_KIN])
@pytest.mark.parametrize("acc", [0.0, 2.0, 3.0, -3.0, -6.0, -9.7])
def test_straight_line_constant_acceleration_is_exact(orc, model, acc):
    """delta = 0: x(t) = x0 + v0 t + a t^2 / 2 along psi0 until the stop at t_s = v0/|a|, then at rest
    v0^2 / (2|a|) from the start.  The discrete scheme reaches this exactly (reading a_x,0 = vdot)."""
    v0, psi0 = np.float32(12.3), np.float32(0.7)
    p = gen(orc, [car(x0=3.0, y0=-4.0, psi0=psi0, v0=v0, acc=(acc,))], n=40, model=model)
    t = times(0.1, 40)
    v0d, a = float(v0), float(np.float32(acc))
    if a < 0:
        ts = v0d / -a
        s = np.where(t < ts, v0d * t + a * t * t / 2, v0d * v0d / (2 * -a))
    else:
        s = v0d * t + a * t * t / 2
    np.testing.assert_allclose(p["x"][0], 3.0 + s * math.cos(float(psi0)), atol=1e-9)
    np.testing.assert_allclose(p["y"][0], -4.0 + s * math.sin(float(psi0)), atol=1e-9)
    np.testing.assert_allclose(p["psi"][0], float(psi0), atol=1e-15)


def test_stopping_distance(orc):
    v0 = float(np.float32(14.0))
    for a in (-3.5, -7.0, -9.7):
        p = gen(orc, [car(v0=v0, acc=(a,))], n=60)
        a = float(np.float32(a))
        assert abs(p["x"][0, -1] - v0 * v0 / (2 * -a)) < 1e-9


@pytest.mark.parametrize("v", [8.0, 12.0, 20.0])
@pytest.mark.parametrize("delta", [0.02, -0.05, 0.1])
def test_one_track_steady_state_yaw_rate(orc, v, delta):
    """At constant speed and steering the linear bicycle model settles at the textbook steady state
    r_ss = v delta / (L + K_us v^2), K_us = m (l_r c_r - l_f c_f) / (L c_f c_r).  The Euler fixed point is the
    continuous equilibrium, so the late yaw increments match it to rounding."""
    m, Iz, lf, lr, cf, cr = (float(x) for x in S.DEFAULT_VEH_PARAMS)
    L = lf + lr
    K = m * (lr * cr - lf * cf) / (L * cf * cr)
    v, delta = float(np.float32(v)), float(np.float32(delta))
    r_ss = v * delta / (L + K * v * v)
    p = gen(orc, [car(v0=v, steer=(delta,))], tau=0.1, n=60, k=5)
    dpsi = np.diff(p["psi"][0]) / float(np.float32(0.1))
    assert abs(dpsi[-1] - r_ss) < 1e-9 * max(1.0, abs(r_ss))


def test_understeer_sign(orc):
    """With l_r c_r > l_f c_f (understeer) the steady yaw rate is below the kinematic v delta / L."""
    v, d = 20.0, 0.05
    p = gen(orc, [car(v0=v, steer=(d,))], n=60)
    r = (p["psi"][0, -1] - p["psi"][0, -2]) / float(np.float32(0.1))
    lf, lr = (float(x) for x in S.DEFAULT_VEH_PARAMS[2:4])
    assert 0 < r < v * float(np.float32(d)) / (lf + lr)


def test_substep_convergence_first_order(orc):
    """Explicit Euler: refining the sub-step 10x shrinks the error ~10x (first order)."""
    objs = [car(v0=11.0, acc=(1.0,), steer=(0.2,))]
    ref = gen(orc, objs, tau=0.1, n=30, k=2000)
    errs = []
    for k in (5, 50):
        p = gen(orc, objs, tau=0.1, n=30, k=k)
        errs.append(np.hypot(p["x"][0] - ref["x"][0], p["y"][0] - ref["y"][0]).max())
    ratio = errs[0] / errs[1]
    assert 5.0 < ratio < 20.0, (errs, ratio)


def test_constant_speed_straight_steps_are_equal(orc):
    p = gen(orc, [car(v0=9.0, psi0=2.0)], n=25)
    d = np.hypot(np.diff(p["x"][0]), np.diff(p["y"][0]))
    np.testing.assert_allclose(d, float(np.float32(9.0)) * float(np.float32(0.1)), rtol=1e-12)


def test_kinematic_model_circle(orc):
    """Kinematic bicycle at constant v and delta: heading grows linearly at r = v cos(beta) tan(delta) / L with
    beta = atan(l_r tan(delta) / L); the centre of gravity stays on a circle of radius v / r (to O(tau^2))."""
    v, d = float(np.float32(10.0)), float(np.float32(0.25))
    lf, lr = (float(x) for x in S.DEFAULT_VEH_PARAMS[2:4])
    L = lf + lr
    beta = math.atan(lr * math.tan(d) / L)
    r = v * math.cos(beta) * math.tan(d) / L
    p = gen(orc, [car(v0=v, steer=(d,))], tau=0.1, n=30, k=50, model=S.MODEL_KIN)
    t = times(0.1, 30)
    np.testing.assert_allclose(p["psi"][0], r * t, atol=1e-9)
    R = v / r
    # circle centre: to the left of the initial course direction beta
    cx, cy = -R * math.sin(beta), R * math.cos(beta)
    rad = np.hypot(p["x"][0] - cx, p["y"][0] - cy)
    assert np.abs(rad - R).max() < 2e-3 * R


def test_low_speed_switch_uses_kinematic_yaw_rate(orc):
    """Below 2 m/s the one-track model is replaced by its kinematic limit: the yaw rate is v cos(beta) tan(delta)/L
    at the current speed."""
    v0, a, d = float(np.float32(3.0)), float(np.float32(-1.0)), float(np.float32(0.1))
    tau, k = float(np.float32(0.1)), 1
    p = gen(orc, [car(v0=v0, acc=(a,), steer=(d,))], tau=0.1, n=25, k=k)
    lf, lr = (float(x) for x in S.DEFAULT_VEH_PARAMS[2:4])
    L = lf + lr
    beta = math.atan(lr * math.tan(d) / L)
    # steps n >= 11: v_n = 3 - 0.1 n < 2 -> psi_{n+1} - psi_n = v_n cos(beta) tan(delta) / L * tau
    for n in range(12, 24):
        v_n = v0 + n * (a * tau)
        dpsi = p["psi"][0, n] - p["psi"][0, n - 1]   # state n+1 minus state n
        assert abs(dpsi - v_n * math.cos(beta) * math.tan(d) / L * tau) < 1e-12


def test_pedestrian_constant_speed(orc):
    speeds, heads = [0.0, 1.3, 3.0], [-1.0, 0.0, 0.5]
    p = gen(orc, [ped(x0=1.0, y0=2.0, psi0=0.3, grid_a=speeds, grid_b=heads)], n=20)
    t = times(0.1, 20)
    for i, v in enumerate(speeds):
        for j, h in enumerate(heads):
            th = float(np.float32(0.3)) + float(np.float32(h))
            row = i * 3 + j
            np.testing.assert_allclose(p["x"][row], 1.0 + float(np.float32(v)) * t * math.cos(th), atol=1e-12)
            np.testing.assert_allclose(p["y"][row], 2.0 + float(np.float32(v)) * t * math.sin(th), atol=1e-12)


def test_pedestrian_acceleration_with_cap(orc):
    """Paper's pedestrian sampling (accelerations, speed cap 2.7 m/s): distance travelled is the closed-form
    integral of a speed that ramps linearly and saturates at the cap or at zero."""
    v0, cap = float(np.float32(1.0)), float(np.float32(2.7))
    accs = [-12.0, -2.0, 0.0, 0.5, 12.0]
    p = gen(orc, [ped(v0=v0, grid_a=accs, grid_b=[0.0], v_max=cap, flags=S.PED_ACCEL_GRID)], n=30, k=3)
    t = times(0.1, 30)
    for i, a in enumerate(accs):
        a = float(np.float32(a))
        if a > 0:
            ts = (cap - v0) / a
            s = np.where(t < ts, v0 * t + a * t * t / 2, v0 * ts + a * ts * ts / 2 + cap * (t - ts))
        elif a < 0:
            ts = v0 / -a
            s = np.where(t < ts, v0 * t + a * t * t / 2, v0 * v0 / (2 * -a))
        else:
            s = v0 * t
        np.testing.assert_allclose(p["x"][i], s, atol=1e-10)


def test_generation_is_deterministic(orc):
    sc = S.intersection11(7, n_acc=5, n_str=5, n_ped_v=3, n_ped_h=3)
    a, b = orc.generate(sc), orc.generate(sc)
    for k in ("x", "y", "psi"):
        assert np.array_equal(a[k], b[k])


def test_rotation_and_translation_covariance(orc):
    """Rotating and translating the initial state rotates and translates every trajectory (the models are
    frame-free)."""
    th, tx, ty = 0.8, 5.0, -7.0
    base = car(x0=0.0, y0=0.0, psi0=0.0, v0=10.0, acc=(-2.0, 1.0), steer=(-0.2, 0.15))
    moved = car(x0=tx, y0=ty, psi0=th, v0=10.0, acc=(-2.0, 1.0), steer=(-0.2, 0.15))
    th = float(np.float32(th))
    p, q = gen(orc, [base]), gen(orc, [moved])
    xr = tx + math.cos(th) * p["x"] - math.sin(th) * p["y"]
    yr = ty + math.sin(th) * p["x"] + math.cos(th) * p["y"]
    np.testing.assert_allclose(q["x"], xr, atol=1e-9)
    np.testing.assert_allclose(q["y"], yr, atol=1e-9)
    np.testing.assert_allclose(q["psi"], p["psi"] + th, atol=1e-12)


@pytest.mark.parametrize("v,delta", [(12.0, 0.1), (20.0, -0.04), (8.0, 0.2)])
def test_one_track_steady_state_sideslip(orc, v, delta):
    """In steady cornering the centre of gravity moves along heading + beta_ss with the textbook sideslip
    beta_ss = delta (l_r - l_f m v^2 / (c_r L)) / (L + K_us v^2).  The chord between two late poses points
    along the course at the mid time, i.e. at (psi_k + psi_k+1)/2 + beta_ss."""
    m, Iz, lf, lr, cf, cr = (float(x) for x in S.DEFAULT_VEH_PARAMS)
    L = lf + lr
    K = m * (lr * cr - lf * cf) / (L * cf * cr)
    v, delta = float(np.float32(v)), float(np.float32(delta))
    beta_ss = delta * (lr - lf * m * v * v / (cr * L)) / (L + K * v * v)
    p = gen(orc, [car(v0=v, steer=(delta,))], tau=0.02, n=300, k=20)
    dx, dy = p["x"][0, -1] - p["x"][0, -2], p["y"][0, -1] - p["y"][0, -2]
    course = math.atan2(dy, dx)
    mid = 0.5 * (p["psi"][0, -1] + p["psi"][0, -2])
    err = (course - mid - beta_ss + math.pi) % (2 * math.pi) - math.pi
    assert abs(err) < 2e-4, (err, beta_ss)


def _linear_bicycle(v, tau):
    m, Iz, lf, lr, cf, cr = (float(x) for x in S.DEFAULT_VEH_PARAMS)
    A = np.array([[-(cf + cr) / (m * v), (cr * lr - cf * lf) / (m * v * v) - 1.0],
                  [(cr * lr - cf * lf) / Iz, -(cf * lf * lf + cr * lr * lr) / (Iz * v)]])
    b = np.array([cf / (m * v), cf * lf / Iz])
    return A, b


def test_one_track_transient_heading_closed_form(orc):
    """At constant speed the (beta, r) recurrence of Eq. EulerVelocity is linear, z_n+1 = (I + tau A) z_n + tau b delta,
    so z_n = z_ss + (I + tau A)^n (z_0 - z_ss) with z_ss = -A^-1 b delta (matrix powers, no stepping), and the
    heading sums r_n tau + rdot_n tau^2 / 2 with rdot_n = (A z_n + b delta)_2."""
    v, d, tau, K, N = float(np.float32(9.0)), float(np.float32(0.15)), float(np.float32(0.1)), 5, 20
    taui = tau / K
    A, b = _linear_bicycle(v, taui)
    zss = -np.linalg.solve(A, b * d)
    M = np.eye(2) + taui * A
    n = np.arange(N * K)
    z = np.array([zss + np.linalg.matrix_power(M, int(k)) @ (-zss) for k in n])
    rdot = (z @ A.T + b * d)[:, 1]
    dpsi = z[:, 1] * taui + rdot * taui * taui / 2
    psi = np.concatenate([[0.0], np.cumsum(dpsi)])[K::K]
    p = gen(orc, [car(v0=v, steer=(d,))], tau=0.1, n=N, k=K)
    np.testing.assert_allclose(p["psi"][0], psi, atol=1e-12)


def test_one_track_transient_lateral_offset_small_angle(orc):
    """Small steering (delta = 1e-4 rad) from heading 0: to first order in delta the lateral position is
    sum_n v tau (psi_n + beta_n) + a_y,n tau^2 / 2, with a_y,n = v (betadot_n-1 + r_n-1) the derivative of the
    lateral velocity (a_y,0 = 0).  The (beta, r) sequence comes from the matrix-power closed form."""
    v, d, tau, K, N = float(np.float32(6.0)), float(np.float32(1e-4)), float(np.float32(0.1)), 5, 12
    taui = tau / K
    A, b = _linear_bicycle(v, taui)
    zss = -np.linalg.solve(A, b * d)
    M = np.eye(2) + taui * A
    n = np.arange(N * K)
    z = np.array([zss + np.linalg.matrix_power(M, int(k)) @ (-zss) for k in n])
    zdot = z @ A.T + b * d
    psi = np.concatenate([[0.0], np.cumsum(z[:, 1] * taui + zdot[:, 1] * taui * taui / 2)])[:-1]
    ay = np.concatenate([[0.0], v * (zdot[:-1, 0] + z[:-1, 1])])
    y = np.cumsum(v * taui * (psi + z[:, 0]) + ay * taui * taui / 2)[K - 1::K]
    p = gen(orc, [car(v0=v, steer=(d,))], tau=0.1, n=N, k=K)
    np.testing.assert_allclose(p["y"][0], y, rtol=1e-6, atol=1e-13)


@pytest.mark.parametrize("v,delta", [(20.0, 0.05), (12.0, -0.12)])
def test_steady_cornering_acceleration_is_centripetal(orc, v, delta):
    """In steady cornering at constant speed the velocity-derivative term of Eq. EulerVelocity is purely
    centripetal (|a| = v r, perpendicular to the velocity), so every sub-step advances by the chord
    v tau sqrt(1 + (r tau / 2)^2) with r = r_ss."""
    m, Iz, lf, lr, cf, cr = (float(x) for x in S.DEFAULT_VEH_PARAMS)
    L = lf + lr
    K = m * (lr * cr - lf * cf) / (L * cf * cr)
    v, delta, tau = float(np.float32(v)), float(np.float32(delta)), float(np.float32(0.1))
    r_ss = v * delta / (L + K * v * v)
    p = gen(orc, [car(v0=v, steer=(delta,))], tau=0.1, n=80, k=1)
    chord = math.hypot(p["x"][0, -1] - p["x"][0, -2], p["y"][0, -1] - p["y"][0, -2])
    assert abs(chord - v * tau * math.sqrt(1 + (r_ss * tau / 2) ** 2)) < 1e-9
