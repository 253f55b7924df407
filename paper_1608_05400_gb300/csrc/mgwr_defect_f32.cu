// Defect instantiations: FP32.
#include "mgwr_defect.cuh"

namespace mgwr {
template cudaError_t launch_defect<float, float>(const float*, const float*, float*,
                                                 const Cx<float>*, size_t, const Cx<float>*,
                                                 const float*, Cx<float>*, const LevelShape&,
                                                 float, unsigned long long*, int, cudaStream_t);

}  // namespace mgwr
