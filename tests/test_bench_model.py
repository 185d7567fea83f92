"""The benchmark's algorithmic-byte model of the two PCG phases (host logic, no GPU)."""
import pytest

import bench


def test_bytes_per_unknown_match_the_stored_fields():
    # FP64: phase A moves z, u', p in and u, v, p out (48 B), phase B r, v in and
    # r, z out (32 B); D, aE, aN of 5 coefficient slots serve 9 conditions in each
    fp64 = bench.alg_bytes_per_dof("fp64")
    assert fp64["phase_a"] == pytest.approx(48 + 24 * 5 / 9)
    assert fp64["phase_b"] == pytest.approx(32 + 24 * 5 / 9)
    assert fp64["phase_a"] + fp64["phase_b"] == pytest.approx(106.6667, abs=1e-3)
    mixed = bench.alg_bytes_per_dof("mixed")
    assert mixed["phase_a"] + mixed["phase_b"] == pytest.approx(53.3333, abs=1e-3)


def test_paired_p_updates_save_two_bytes_per_unknown_in_fp32():
    # every second iteration: p read and written, plus the older direction read
    one = bench.alg_bytes_per_dof("mixed", p_period=1)
    two = bench.alg_bytes_per_dof("mixed", p_period=2)
    assert one["phase_a"] - two["phase_a"] == pytest.approx(2.0)
    assert one["phase_b"] == two["phase_b"]


def test_rebuilt_diagonal_drops_one_coefficient_array_from_phase_a():
    base = bench.alg_bytes_per_dof("mixed", p_period=2)
    drec = bench.alg_bytes_per_dof("mixed", p_period=2, diag_rebuilt=True)
    assert base["phase_a"] - drec["phase_a"] == pytest.approx(4 * 5 / 9)
    assert base["phase_b"] == drec["phase_b"]
    assert bench.diag_rebuilt(10604322) and not bench.diag_rebuilt(604322)
    assert not bench.diag_rebuilt(600604183) and not bench.diag_rebuilt(3014062)
