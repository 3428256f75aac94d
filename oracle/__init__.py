"""CPU FP64 oracle for tensor-network coset decoding (arXiv 2310.10722).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only the test
suite, the smoke check and the CPU-baseline leg of the benchmark may use it.  It shares
no code with the CUDA path; the only common module is ``td_inputs`` (problem
generators and the seeded sampler, which hold none of the decoder's arithmetic).

Contents (each function cites the passage of the paper it follows):
  gf2      -- linear algebra over F_2 (rank, solve, kernel) used by the exact methods.
  exact    -- p_{m,L} of Sec. 2.4 computed exactly three ways:
                brute_force_table   sum over all 2^n error patterns;
                generator_sum       sum over a coset of the kernel (Sec. 3.2);
                transfer_matrix     untruncated layer-by-layer contraction (Sec. 4 without
                                    truncation), and its exact gradient.
  pauli    -- the general optimal decoder of Sec. 2.3 over all 4^n Paulis.
  su       -- the approximate method of Sec. 4: sweep a PEPS through the layered network,
              simple-update truncation to chi after every gate, final boundary-MPS
              contraction with chi_mps, then coset log-probabilities; and the
              gradient of its total log P by the affine identity in each rate.
  reverse  -- the gradient of su's total log P by reverse-mode differentiation through
              every step of the sweep, truncations included.
  frozen   -- the "frozen projector" reading of the gradient, kept only to show that it
              is not the gradient (tests/test_oracle_grad.py).
All arithmetic is float64.  Pins are in tests/test_oracle_*.py.
"""
