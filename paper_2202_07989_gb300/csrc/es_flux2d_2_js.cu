// Fused 2D stage kernels of the 2-species case with the WENO-JS dissipation, in both
// compute types and every fused tile shape.
#include "es_flux2d_impl.cuh"

namespace es {
ES_FLUX2D_INSTANTIATE(2, 1)
}  // namespace es
