// k_aos_va.cu -- instantiates one group of the AOS line-solver
// variants (aos_solver.cuh) so the groups compile in parallel.
#include "aos_solver.cuh"

namespace kz {
namespace aos {
KZ_AOS_VARIANTS_A(KZ_AOS_INSTANTIATE)
}  // namespace aos
}  // namespace kz
