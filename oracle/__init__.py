"""Oracle for the fixed-sector fermionic state-vector path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import anything from this package.  The
product path (the CUDA library and its Python binding) never calls it, and
shares no code, tables or constants with it.

Plain, slow, obviously-correct complex128 NumPy/SciPy code written from the
paper: string addresses (§3.1), number-operator-sum and diagonal-Coulomb
evolution (§3.2.1, §3.2.2), orbital rotations by minor determinants (§2.3)
and by Givens rotations (§3.2.3), the LUCJ ansatz (§4.3, §4.5.1) and its
gradient, the remaining gates of Table 1, Trotter-Suzuki time evolution
of double-factorized and diagonal-Coulomb Hamiltonians, the action of a
molecular Hamiltonian on a state, and sampling configurations from a state
or a Slater determinant.  Each function is pinned by tests that do not reuse it: a dense
Jordan-Wigner construction with matrix exponentials (`bruteforce`), the
Slater-determinant closed form (§2.4), the group-homomorphism identities of
§2.3, the gate equivalences listed after Table 1, the state sizes printed in
§1, §5.2 and §6.1, finite differences for the gradient, the convergence
order of the product formulas against exact evolution, and for the samplers
the chain rule summed over pick orders against |det U[I, occ]|^2 and sample
frequencies against the exact distributions.
"""

from .strings import strings, address_map, occupations, excite
from .gates import (dims, hartree_fock, apply_num_op_sum_evolution,
                    apply_diag_coulomb_evolution, diag_coulomb_angle,
                    diag_coulomb_angle_entry, rotated_string,
                    minor_matrix, minor_matrix_row, rotated_amplitude,
                    apply_orbital_rotation,
                    apply_orbital_rotation_minors, apply_orbital_rotation_givens,
                    apply_givens, givens_matrix, givens_decomposition,
                    slater_from_hf)
from .lucj import (lucj_forward, lucj_vjp, transition_one_body,
                   expm_frechet_adjoint)
from .trotter import (apply_num_interaction, apply_num_num_interaction,
                      apply_givens_rotation, apply_tunneling_interaction,
                      apply_quad_ham_evolution, product_formula,
                      simulate_trotter_double_factorized, simulate_trotter_diag_coulomb)
from .operator import apply_molecular_hamiltonian
from .sampling import sample_state, sample_slater_spin, chain_rule_probability
