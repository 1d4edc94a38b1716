"""Plain CPU oracle of the TNMCMC slice update, in FP64.

This package is test infrastructure. It is a slow, literal restatement of the
paper's method used to check the CUDA path, and only ``tests/``,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference legs
may import it. The product library never calls it and has no CPU fallback.

Modules:
  philox        Philox4x32-10 draws of the method (fixed line, site, MH uniforms)
  model         energies, slice geometry, held fields, Boltzmann factors
  bmps          boundary-MPS environments (MPO x MPS + LQ/SVD truncation), sampler
  update        one slice update (proposal + MH) and the sweep schedule
  exact         brute-force enumeration used to pin the above on tiny cases
  observables   overlap q and the integrated autocorrelation time
  arnet         the masked-convolution autoregressive proposal network
"""
