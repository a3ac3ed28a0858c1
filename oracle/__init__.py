"""Plain, slow, FP64 CPU oracle for composed split-operator propagation in the
diabatic representation (Roulet, Choi, Vanicek, arXiv:1903.04946).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
It shares no code with the CUDA library: it has its own composition
coefficients (Sec. II D-F), its own radix-2 FFT and direct DFT (Sec. II G),
its own potential exponentials (Sec. II H), its own propagation loop and
observables (Sec. II A).  Each function names the passage it follows.

Modules
-------
coefficients   recursive triple-jump / Suzuki coefficients, expansion to
               splitting coefficients, pruning, unique-value index arrays
fourier        iterative radix-2 FFT along one axis, direct DFT, N-d helpers
operators      grids, momenta, kinetic phases, potential exponentials
propagate      split-operator sequences (VT, TV, VTV, TVT and compositions)
observables    norm, populations, inner product, symplectic form, energy
brute          dense grid Hamiltonian and exact exp(-iHt) on tiny grids
"""
