// Flux kernels of the 3D, 1-species case with the WENO-MR dissipation, in both compute
// types and every tile shape (one translation unit per case keeps the build parallel).
#include "es_flux_impl.cuh"

namespace es {
ES_FLUX_INSTANTIATE(3, 1, 0)
}  // namespace es
