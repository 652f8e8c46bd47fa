"""The seeded input generators: determinism and the FFT synthesis of waves."""
import math

import numpy as np

from paper_1805_03442_gb300 import inputs


def test_waves_fft_equals_direct_sum():
    N, L = 256, 3.0
    modes = inputs.random_phase_modes(5, np.array([1.0, 0.5 - 0.2j, 2.0, 0.1j]), 6, 3, 1e-2, m_step=7)
    U = inputs.waves_1d(1.4, N, L, (1.0, 1.0, 1.1), modes)
    x = inputs.cell_centres(N, L)
    pert = np.zeros((4, N))
    for md in modes:
        for f in range(4):
            pert[f] += np.real(md.scale * md.shape[f] * np.exp(1j * 2 * math.pi * md.m / L * x))
    ref = inputs.prim_to_cons(1.4, 1.0 + pert[0], [pert[1]], 1.0 + pert[2], 1.1 + pert[3])
    assert np.allclose(U, ref, rtol=1e-13, atol=1e-15)


def test_generators_are_seeded():
    a = inputs.random_states(2, 100, seed=3, smooth=True)
    b = inputs.random_states(2, 100, seed=3, smooth=True)
    assert np.array_equal(a, b)
    r1 = inputs.sweep_runs(1, 10)
    r2 = inputs.sweep_runs(1, 10)
    assert r1 == r2
