"""CPU oracle for the wall-corrected RPY rigid-multiblob hot path.

TEST INFRASTRUCTURE.  Plain, slow, FP64 implementations of what the CUDA
library computes, written from the paper (Sprinkle, Balboa Usabiaga,
Patankar, Donev, "Large Scale Brownian Dynamics of Confined Suspensions of
Rigid Particles"), each function citing the passage it follows.  Only tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline / reference leg may
import anything from here; the product package never does.  The oracle shares
no code with the CUDA path; both take inputs from paper_1709_02410_gb300.synth.

Parity status per function (pins live in tests/test_oracle_*.py):
  mobility (M F, dense M, pair blocks)  pinned: closed-form near-wall self
      mobility, free-space RPY limit, Blake no-slip and reciprocity,
      symmetry, SPD, r = 2a continuity, far-field decay
  gradient / divergence                 pinned: central finite differences,
      horizontal translation invariance, divergence-free free-space RPY
  rigid K, K^T, quaternions, Rotate      pinned: adjointness, rigid motion,
      eq. (rotate) expansion, norm preservation
  block preconditioner                   pinned: dense Schur solve, one body
  Lanczos M^{1/2} W                      pinned: dense sqrtm, covariance
  GMRES saddle solve                     pinned: dense Schur form (eq. sysDense)
  RFD drift                              pinned: exact divergence in the mean
  Philox4x32-10 / Box-Muller             pinned: published known-answer vectors
  T-S, EM-T, EM-RFD, T-T steps           pinned: deterministic orders (kT = 0);
      drift consistency -- the mean step equals the Ito drift
      kT d_Q.(Psi N Psi^T) of App. B (eq. quatLangevin) at two bodies, from
      a dense N and finite differences that share no code with the steps,
      and a variant with D^S or D^F negated fails it
"""
