"""CPU oracle for the sliced sparse-state contraction and its sampler.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
the tests, the smoke check and the benchmark's CPU-baseline leg call it.  It is
plain, slow, complex128 NumPy written from the paper's definitions:

* ``statevector``   -- O1: apply the circuit's gates in time order to |0...0>,
                       cut edges acting as |v><v| projectors (the edge-breaking
                       matrix E of the Method section, generalised to value v);
* ``network``       -- O2: an independent tensor-network builder contracted
                       pairwise with ``numpy.tensordot``, one group at a time;
* ``metrics``       -- fidelity, the fidelity estimate, linear and
                       logarithmic XEB, entropies, the Porter-Thomas check,
                       the GPU-efficiency formula;
* ``sampler``       -- the group sampler and its Philox-4x32-10 generator.

The oracle shares no code with the CUDA path; both read the seeded inputs of
``circuit_inputs``.
"""
from .statevector import (statevector, sliced_statevector, sparse_state_from_vector,
                          brute_force_state, bitstring_index)
from .network import network_amplitudes
from .metrics import (fidelity, f_estimate, companion_factor, linear_xeb, expected_group_sampler_xeb,
                      porter_thomas_ks, gpu_efficiency, normalised_probabilities, log_xeb, entropy,
                      entropy_from_samples, group_sampling_law, EULER_GAMMA, expected_subgroup_xeb,
                      subset_fidelity)
from .sampler import philox4x32_10, sample_groups, sample_groups_mcmc
