"""Oracle: a plain, slow, complex128 CPU restatement of GOCP ADAPT-VQE.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The product path (the CUDA library and its Python binding) never does, and
this package never imports the product: the two share no code.  Both sides
take their seeded inputs from ``synth``, which holds no method arithmetic.

Every function follows the paper's definitions literally, in the paper's
order, in float64 / complex128 (the paper fixes no precision):

  * ``mapping``     Eq. (2) fermionic Hamiltonian -> Eq. (3) Pauli sum under
                    Jordan-Wigner and Bravyi-Kitaev (Sec. II.A).
  * ``pool``        spin-conserving singles + doubles pool (Table II counts).
  * ``gocp``        non-commutativity graph + Largest-First colouring
                    (Sec. III.A, Algorithm 1).
  * ``statevector`` term-by-term Pauli-sum application, the O(5) Taylor chain
                    (Eq. 5, Eq. 6), the Rayleigh quotient (Eq. 1), pool
                    gradients (Eq. 4) and forward-mode dE/dtheta.
  * ``adapt``       the ADAPT-VQE loop (Sec. II.B).
  * ``parallel``    the same statevector functions on slices of rows or of
                    pool operators in spawned worker processes (no
                    arithmetic of its own), for full-size checks and timing.

Pauli convention: a term (x, z, phase, c) is c * i**phase * X^x Z^z with x, z
bit masks (bit j = qubit j); it maps |b> to c * i**phase * (-1)**popc(b & z)
|b ^ x>.  The pins that tie each function to something other than itself are
in ``tests/test_oracle_*.py``; every function here is pinned.
"""
