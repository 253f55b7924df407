// Defect instantiations: FP64 iterate (FP64 or FP32 output).
#include "mgwr_defect.cuh"

namespace mgwr {
template cudaError_t launch_defect<double, double>(const double*, const double*, double*,
                                                   const Cx<double>*, size_t, const Cx<double>*,
                                                   const double*, Cx<double>*, const LevelShape&,
                                                   double, unsigned long long*, int, cudaStream_t);
template cudaError_t launch_defect<double, float>(const double*, const double*, float*,
                                                  const Cx<double>*, size_t, const Cx<double>*,
                                                  const double*, Cx<double>*, const LevelShape&,
                                                  double, unsigned long long*, int, cudaStream_t);

}  // namespace mgwr
