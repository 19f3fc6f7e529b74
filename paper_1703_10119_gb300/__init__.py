"""GB300-native library for the Dufort-Frankel hygrothermal wall update.

Hot path of Gasparin, Berger, Dutykh & Mendes, "An improved explicit scheme
for whole-building hygrothermal simulation" (arXiv:1703.10119): the
three-level DF update of coupled nonlinear heat and vapour-pressure
diffusion in porous walls, batched over many ragged walls.

Submodules: ``hygro`` (binding of the C ABI in include/hygro.h), ``build``
(nvcc build of libhygro.so for sm_103a), ``workloads`` (seeded synthetic
inputs). Importing the package loads nothing; the binding loads the CUDA
library on first use and raises if it is missing.
"""
