"""FP64 CPU oracle of the block-structured Euler update, plus exact solutions.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs may import anything here.  Nothing in this
package is shared with, or imported by, the CUDA library.

Parity status per function (what pins it, see tests/test_oracle_*.py):
  prim_from_cons  pinned: round trip with the stated initial data, floors.
  mc_slope        pinned: hand-computed cases of the MC definition, TVD bound.
  hllc            pinned: consistency F(U,U)=F(U), stationary / moving contacts
                  resolved exactly, supersonic upwinding, mirror symmetry,
                  Rankine-Hugoniot across each wave of the fan, integral
                  consistency of the fan.
  fill/stage/step pinned: Sod shock tube vs the exact Riemann solution with
                  first-order convergence, Sedov blast vs the self-similar
                  radius, round-off conservation on periodic domains, block
                  decomposition invariance (bitwise), 1-D rows bitwise equal,
                  axis permutation, corner-guard independence.
  compute_dt      pinned: closed form on uniform states.
"""
