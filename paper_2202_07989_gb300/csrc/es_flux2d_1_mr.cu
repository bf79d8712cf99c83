// Fused 2D stage kernels of the single-species case with the WENO-MR dissipation, in both
// compute types and every fused tile shape.
#include "es_flux2d_impl.cuh"

namespace es {
ES_FLUX2D_INSTANTIATE(1, 0)
}  // namespace es
