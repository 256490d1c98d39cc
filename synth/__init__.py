"""Seeded synthetic fields shaped like the workloads of the ProAICD evaluation.

This module is the only code shared by the CPU oracle and the CUDA path: it
draws random fields and holds none of the compressor's arithmetic.  The paper's
datasets (CESM, Miranda, SCALE, S3D, JHTDB; evaluation section, dataset table)
are not available, so each recipe below stands in for one of them with the
same shape and a similar statistical character.

Recipes (all seeded with numpy PCG64, generated in float64 then cast):

* ``gaussians``  -- sum of random 3-D Gaussian blobs plus N(0, sigma) noise.
* ``grf``        -- spectral Gaussian random field with a Kolmogorov spectrum
                    (|u_hat(k)| ~ k^-11/6 in 3-D, k^-4/3 in 2-D, i.e. a shell
                    energy spectrum E(k) ~ k^-5/3), random phases, rescaled to
                    [-1, 1] (turbulence stand-in for S3D / JHTDB).
* ``climate``    -- zonal bands cos(lat) sin(k lon + phi) for three wavenumbers
                    times a lognormal small-scale factor (Miranda-shaped stand-in
                    for the CESM / SCALE climate fields).
* ``polynomial`` -- low-degree polynomial fields for the interpolant pins.
"""
from .fields import (gaussians, grf, climate, polynomial, random_field,
                     config_field, CONFIGS)

__all__ = ["gaussians", "grf", "climate", "polynomial", "random_field",
           "config_field", "CONFIGS"]
