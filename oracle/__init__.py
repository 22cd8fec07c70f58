"""CPU oracle for Ozaki-scheme density-matrix purification.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, float64 CPU statement
of what the GPU path computes, written from the paper (Dawson, Domke, Nakajima,
Ozaki, "Reducing Numerical Precision Requirements in Quantum Chemistry
Calculations", arXiv 2407.13299) and the purification method it cites (Palser
and Manolopoulos 1998). Only the tests, the package's `smoke()` self-check and
the benchmark's CPU-baseline leg may import it. The library never calls it: the
product path fails loudly when its CUDA extension is missing.

It shares no code with the CUDA path. Its inputs come from `synth`, which draws
random numbers and holds none of the method's arithmetic.

Modules
  ozaki    -- power-of-two scaling, digit split, level sums, FP64 recombination
              (Sec. "Ozaki Scheme", Fig. 2)
  purify   -- Gershgorin bounds, initial guess, canonical purification loop,
              stopping rules and error metrics (Sec. "Density Matrix
              Purification", "Implementation Details", "Error Evaluation
              Criteria")
  adjoint  -- reverse mode through the purification iterations
  variants -- SP2 and TRS4 purification (TRS4 is the algorithm the paper runs
              through NTPoly, Sec. "Implementation Details")
  foe      -- Chebyshev Fermi-operator expansion at finite electronic
              temperature (the finite-temperature method of Sec. "Introduction")

Parity status per function is stated in each module header.
"""

from . import adjoint, foe, ozaki, purify, variants  # noqa: F401
