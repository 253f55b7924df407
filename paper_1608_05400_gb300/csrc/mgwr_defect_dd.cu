// Defect instantiation: double-float iterate, FP32 output (outer defect of the
// mixed refinement).
#include "mgwr_defect.cuh"

namespace mgwr {
template cudaError_t launch_defect<dd, float>(const dd*, const dd*, float*, const Cx<dd>*, size_t,
                                              const Cx<dd>*, const dd*, Cx<dd>*, const LevelShape&,
                                              dd, unsigned long long*, int, cudaStream_t);
}  // namespace mgwr
