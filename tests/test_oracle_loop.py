"""Oracle pins: the closed loop (integrator, modal mirror, one-step delay) and
its residual statistics, against closed forms."""
import numpy as np

from oracle import geometry, loop, modal

N, NM = 32, 10


def _basis():
    return modal.modal_basis(N, 0.2, NM), geometry.pupil_mask(N, 0.2).astype(np.float64)


def test_stats_closed_forms():
    amp = geometry.pupil_mask(N, 0.0).astype(np.float64)
    assert loop.residual_stats(amp, np.zeros((N, N)), 0.5) == (0.0, 1.0)
    rms, sr = loop.residual_stats(amp, np.full((N, N), 2.7), 0.5)      # pure piston
    assert rms < 1e-12 and abs(sr - 1.0) < 1e-12
    # +a on the left half of the (left-right symmetric) pupil, -a on the right:
    # piston-free, RMS a; the field sums to cos(a k) over the pupil
    a, k = 0.9, 0.4
    ph = np.where(np.arange(N)[None, :] < N // 2, a, -a) * np.ones((N, 1))
    rms, sr = loop.residual_stats(amp, ph, k)
    assert abs(rms - a) < 1e-12 and abs(sr - np.cos(a * k) ** 2) < 1e-12


def test_zero_gain_leaves_the_atmosphere():
    B, amp = _basis()
    rng = np.random.default_rng(1)
    phases = [rng.standard_normal((N, N)) * amp for _ in range(4)]
    st, cmds, resid = loop.run_loop(phases, amp, B, lambda r: np.ones(NM), 0.0, 0.0, 0.7)
    assert np.all(cmds == 0.0) and np.array_equal(resid, phases[-1])
    for k, p in enumerate(phases):
        assert np.allclose(st[k], loop.residual_stats(amp, p, 0.7), rtol=0, atol=1e-15)


def test_ideal_sensor_follows_the_scalar_recursion():
    """A static aberration in the modal space, a sensor returning its exact
    modal projection: c_k = c* (1 - rho^(k+1)), rho = 1 - leak - gain,
    c* = gain a / (gain + leak); the residual is B^T (a - c_{k-1}).  Pins the
    sign of the correction, the one-step delay and the leak."""
    B, amp = _basis()
    mask = amp > 0
    a = np.linspace(0.5, -0.4, NM)
    phi = loop.dm_shape(B, a)

    def sensor(r):
        return modal.project(B, r, mask)

    for gain, leak in ((0.5, 0.0), (0.3, 0.05), (1.0, 0.0)):
        st, cmds, _ = loop.run_loop([phi] * 12, amp, B, sensor, gain, leak, 1.0)
        rho = 1.0 - leak - gain
        cstar = gain * a / (gain + leak)
        for k in range(12):
            ref = cstar * (1.0 - rho ** (k + 1))
            assert np.max(np.abs(cmds[k] - ref)) < 1e-10, (gain, leak, k)
            prev = cmds[k - 1] if k else np.zeros(NM)
            rms_ref, sr_ref = loop.residual_stats(amp, loop.dm_shape(B, a - prev), 1.0)
            assert abs(st[k][0] - rms_ref) < 1e-10 and abs(st[k][1] - sr_ref) < 1e-10


def test_dm_shape_is_the_modal_sum():
    B, _ = _basis()
    c = np.arange(NM, dtype=np.float64) - 3.0
    ref = np.zeros((N, N))
    for j in range(NM):
        ref += c[j] * B[j]
    assert np.max(np.abs(loop.dm_shape(B, c) - ref)) < 1e-12
