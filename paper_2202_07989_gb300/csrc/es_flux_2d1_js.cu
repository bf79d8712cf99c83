// Flux kernels of the 2D, 1-species case with the WENO-JS dissipation, in both compute
// types and every tile shape (one translation unit per case keeps the build parallel).
#include "es_flux_impl.cuh"

namespace es {
ES_FLUX_INSTANTIATE(2, 1, 1)
}  // namespace es
