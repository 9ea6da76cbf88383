"""FP64 CPU oracle for the finite-difference LLG right-hand side.

TEST INFRASTRUCTURE ONLY.  Nothing in the solver library may import,
call or link this package: only the tests, `__graft_entry__.smoke()` and
the `cpu_baseline` / reference leg of `bench.py` use it.  It shares no
code with the CUDA path (no kernels, helpers, tables or constants); the
only common module is `synth`, which builds seeded inputs.

It is plain, slow and written to be checked by eye against the paper
(arXiv 2406.16064, MicroMagnetic.jl):

  newell     Newell demag tensor (Sec. "Magnetostatic energy", Eqs. 6-8)
  demag      demag field as a direct sum (Eq. 8) or an FFT convolution
  fields     exchange (Eqs. 2-5), interfacial DMI (Eq. 14), uniaxial and
             cubic anisotropy, Zeeman, energies, LL right-hand side
  integrate  adaptive Dormand-Prince RK45 with projection to |m|=1
  neb        geodesic nudged elastic band (Sec. "Miscellaneous")
  minimize   steepest descent with Barzilai-Borwein steps (Sec. "Steepest
             descent energy minimization")
  cayley     fixed-step classical Runge-Kutta with projection and on the
             Cayley-transform variable (Sec. "Cayley transform")
  potential  the demag field through the magnetic scalar potential (the
             three-forward, one-inverse transform variant named in Sec.
             "Magnetostatic energy")

All arithmetic is float64.  Parity status of every function is listed in
its module header.
"""
