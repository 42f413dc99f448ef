"""The seeded input generator (CPU)."""
import numpy as np

from paper_2109_04528_gb300 import inputs


def test_sampling_matrix_is_exactly_hermitian_and_structured():
    # O = [[P, Q], [conj Q, conj P]] in block layout, bit for bit
    for O in (inputs.lossy_squeezed(7, 3).O, inputs.product_state(5, 2).O, inputs.config_n8().O,
              inputs.two_mode_squeezed_vacuum(0.7).O):
        n = O.shape[0] // 2
        assert np.array_equal(O, O.conj().T)
        assert np.array_equal(O[n:, n:], O[:n, :n].conj())
        assert np.array_equal(O[n:, :n], O[:n, n:].conj())


def test_sampling_matrix_is_the_inverse_to_rounding():
    inst = inputs.lossy_squeezed(10, 5, (0.3, 0.8), 0.5)
    direct = np.eye(20) - np.linalg.inv(inst.sigma)
    assert np.max(np.abs(inst.O - direct)) <= 1e-14 * np.max(np.abs(direct))


def test_seeded_inputs_repeat():
    a = inputs.config_single(12).O
    b = inputs.config_single(12).O
    assert np.array_equal(a, b)
