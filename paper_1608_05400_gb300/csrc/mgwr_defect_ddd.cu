// Defect instantiation: double-float iterate, double-float output (double-float
// cycles and the outer defect of MGWR_DD).  A translation unit of its own so that
// the two double-float instantiations compile in parallel.
#include "mgwr_defect.cuh"

namespace mgwr {
template cudaError_t launch_defect<dd, dd>(const dd*, const dd*, dd*, const Cx<dd>*, size_t,
                                           const Cx<dd>*, const dd*, Cx<dd>*, const LevelShape&,
                                           dd, unsigned long long*, int, cudaStream_t);
}  // namespace mgwr
