// Flux kernels of the 2D, 2-species case with the WENO-MR dissipation, in both compute
// types and every tile shape (one translation unit per case keeps the build parallel).
#include "es_flux_impl.cuh"

namespace es {
ES_FLUX_INSTANTIATE(2, 2, 0)
}  // namespace es
