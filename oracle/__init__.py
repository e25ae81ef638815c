"""FP64 CPU oracle for the TD-aGW kernel contraction, commutator and RK4 propagation.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute
anything in this package: only the tests, the smoke check and the CPU-baseline leg of the
benchmark use it.  It shares no code with the CUDA library and imports nothing from it;
its inputs come from ``workloads`` (parameters only) or are passed in explicitly.

Every function follows a passage of arXiv:2502.05635 (cited by section / equation) in
plain numpy/scipy complex128, without blocking, fusion or reordering beyond the written
definition.  Where the paper is silent or garbled, the reading taken is stated at the
function.  Modules:

  model      tight-binding stand-in for the first-principles bands: eigenpairs,
             dipoles (finite-difference Berry connection), velocity
  kernel     screened interaction W(q), its q=0 cell average, the dense direct kernel, the
             optional exchange term, the K^diag / K^off split (strict diagonal or k = k'
             blocks), and an FFT form of K.x (an identity of this kernel)
  lowrank    truncated SVD of K^off, the low-rank apply, R^2 and Eckart-Young error
  channel    channel-wise truncated SVD (dense diagonal channels) and its apply
  hhg        high-harmonic spectrum of a recorded current
  propagate  pulses, the TD-aGW right-hand side, classical RK4, observables
"""
