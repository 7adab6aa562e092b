"""CPU oracle for the mixed real/momentum-space two-site DMRG hot path (arXiv:1512.03318).

TEST INFRASTRUCTURE ONLY. Nothing in the product package imports, links or runs this
package; only tests, the smoke check and the bench's CPU-baseline leg use it. It shares no
code with the CUDA path: its inputs come from the seeded generators in `synth`, and its
expected values come from its own arithmetic (complex128 / float64 numpy).

Modules
  model      -- many-body Hamiltonians by direct operator application (exact
                diagonalisation): real space (Sec. IV.C, Eq. H_real) and mixed real/momentum
                space (Sec. IV.D, Eqs. H_kin and H_k_int); free-fermion closed form.
  mpo        -- finite-state-machine MPO construction (Sec. IV.A-B, Eq. M_example) with
                momentum-labelled nodes and trimming (Sec. IV.D), real and mixed basis.
  dmrg       -- dense (symmetry-free) two-site DMRG with Lanczos and SVD truncation
                (standard DMRG, refs. W92/S2005/S2011 of the paper).
  blocksparse-- charge tables and the block-sparse H_eff / environment update restated in
                plain loops over charge blocks, with the flat memory layout.

Parity status: every function is pinned by tests against exact diagonalisation, closed
forms, brute force or invariants; see the tests named in each module docstring.
"""
