"""Oracle for full-sky Taylor lensing (Naess & Louis 2013) -- TEST INFRASTRUCTURE.

A plain, slow, FP64 CPU implementation of what the GPU library computes, written
from the paper's Sec. II and from textbook definitions (HEALPix geometry of
Gorski et al. 2005; spin-weighted harmonics of Goldberg et al. 1967). Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use it.
It shares no code with the GPU path and never imports it; the product path must
never import it.

Modules:
  healpix  -- RING-scheme ring table, pix2ang, ang2pix
  sht      -- ctypes wrapper over sht.c: spin-weighted lambda and its theta
              derivatives, per-ring Fourier coefficients, direct point sums
  lens     -- derivative-map synthesis, deflection, geodesic displacement,
              pixel-relative Taylor sum (Eq. 4) and polarisation rotation
"""
