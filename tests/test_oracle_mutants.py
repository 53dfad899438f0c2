"""Planted mistakes: each deliberately broken build of the oracle (the
ORACLE_MUTANT hooks in oracle/fmm_oracle.c) must fail at least one of the
pins, which shows the pins are sharp enough to catch that kind of error.
CPU only; the mutants are compiled into a temporary directory."""
import pytest

import oracle
import test_oracle_accel as accel
import test_oracle_m2p as m2p
import test_oracle_ops as ops
import test_oracle_orders as orders
import test_oracle_solve as solve

MUTANTS = {
    1: "M2L with R = source - target (sign of odd orders flipped)",
    2: "M2L without the 1/alpha! factor",
    3: "L2L with the displacement reversed",
    4: "interaction list also takes the near neighbours",
    5: "near field without the self cell",
    6: "near-field pair force pointing away from the mass",
    7: "final-stage M2P without the (-1)^|alpha| factor",
    8: "multipole and local order limits applied to the wrong sides",
    9: "P2M with the cells at their lower corners instead of their centres",
    10: "M2M without the binomial coefficients",
    11: "L2P without the 1/beta! factor",
    12: "5-point stencil with its outer weights' signs flipped",
    13: "stencil transpose with a one-sided edge weight of the wrong sign",
    14: "adjoint chain's L2P^T without the 1/beta! factor",
    15: "gradient of L2P with the undifferentiated factorials",
    16: "near field over the face neighbours only (edge and corner boxes dropped)",
    17: "analytic force's adjoint with the transposed pair force reversed",
    18: "M2P gradient reading D_alpha instead of D_{alpha + e_q}",
}

# Cheap single-operator pins first: a mutant's battery stops at the first pin
# that fails.
PINS = [
    ops.test_p2m_closed_forms,
    ops.test_m2m_equals_direct_p2m_about_parent,
    ops.test_l2p_closed_form,
    ops.test_fd_stencils_exact_on_polynomials,
    ops.test_fd_adjoint_is_transpose,
    ops.test_m2l_converges_geometrically,
    ops.test_l2l_then_l2p_is_exact,
    solve.test_converges_to_direct_sum_in_p,
    solve.test_point_mass_closed_form,
    lambda o: solve.test_equals_direct_sum_when_all_boxes_are_near(o, (8, 8, 8), 4),
    accel.test_accel_converges_to_direct_in_p,
    accel.test_direct_pair_forces_obey_the_third_law,
    m2p.test_m2p_converges_and_beats_m2l_l2p,
    orders.test_monopole_only_far_field_ignores_mass_moved_inside_boxes,
    orders.test_order_zero_locals_give_a_constant_far_field_per_box,
    solve.test_adjoint_chain_is_transpose,
    accel.test_adjoint_of_the_analytic_force_is_its_transpose,
    accel.test_m2p_gradient_is_the_derivative_of_m2p,
]


def _failures(orc, first=False):
    failed = []
    for pin in PINS:
        try:
            pin(orc)
        except AssertionError:
            failed.append(getattr(pin, "__name__", "lambda"))
            if first:
                break
    return failed


def test_battery_passes_on_the_oracle(orc):
    assert _failures(orc) == []


@pytest.mark.parametrize("k", sorted(MUTANTS))
def test_pins_catch_planted_mistake(tmp_path, k):
    path = oracle.build(str(tmp_path / f"liboracle_mutant{k}.so"), mutant=k, force=True)
    mutant = oracle.Oracle(oracle.load(path))
    failed = _failures(mutant, first=True)
    print(f"mutant {k} ({MUTANTS[k]}): caught by {failed[0] if failed else 'nothing'}")
    assert failed, f"no pin caught mutant {k}: {MUTANTS[k]}"
