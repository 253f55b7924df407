// Defect instantiations: FP64 iterate (FP64, FP32 or double-float output).
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
// FP64 defect held in double-float: the anchor of MGWR_MIXED's carried outer
// defects (launch_defect_update)
template cudaError_t launch_defect<double, dd>(const double*, const double*, dd*,
                                               const Cx<double>*, size_t, const Cx<double>*,
                                               const double*, Cx<double>*, const LevelShape&,
                                               double, unsigned long long*, int, cudaStream_t);

}  // namespace mgwr
