"""CPU reference oracle for the differentiable-MPS VQE hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) imports, links or calls anything in this package; only
`tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / `--impl reference`
legs of `bench.py` use it.

It is a plain, slow, float64 / complex128 restatement of the paper's method
(arXiv:2211.07983), written for checking by eye against the paper:

* `pauli`      Pauli-string algebra, Jordan-Wigner Hamiltonian (Sec. 2, Eqs.
               ham-pbc, expect-val), term merging, canonical order, sweep batches.
* `fermion`    independent occupation-number (second-quantised) matrices, used
               only to pin `pauli` (no Jordan-Wigner inside).
* `ansatz`     UCCSD excitation generators -> nearest-neighbour gate list
               (Sec. 2, UCC ansatz and Trotter "V-shaped blocks"; Sec. 3, gate
               fusion).
* `mps`        MPS simulator (Sec. 3, Eqs. mps, hf, rightcanonicalcondition,
               two-qubit gate update, paulistringexp) and the exact reverse-mode
               gradient of the truncated forward pass (Sec. 4, Eqs.
               expecgrad / circuitevolvegrad; App. A complex AD rules).
* `statevector` dense brute-force simulator (Sec. 1 "brute force method") with
               Algorithm 1 on a state vector; pins `mps` for small n.
"""
