// The learned proposal's instances of the finder (find_kernel.cuh): compiled apart from the plain
// ones, so that each kind's register allocation is its own.
#include "find_kernel.cuh"

namespace kfgb {

#define KF_LEARNED_INSTANCE(KC, FEAT)                                                                  \
  template int find_occupancy<KC, true, FEAT>(int, size_t, int*);                                      \
  template void find_launch_kernel<KC, true, FEAT>(const DevGeom&, const DevMat&, const FindArgs&, int, int, \
                                                   size_t, cudaStream_t);
KF_LEARNED_INSTANCE(1, 0) KF_LEARNED_INSTANCE(1, kFeatAll) KF_LEARNED_INSTANCE(2, 0) KF_LEARNED_INSTANCE(2, kFeatAll)
KF_LEARNED_INSTANCE(4, 0) KF_LEARNED_INSTANCE(4, kFeatAll) KF_LEARNED_INSTANCE(6, 0) KF_LEARNED_INSTANCE(6, kFeatAll)
KF_LEARNED_INSTANCE(8, 0) KF_LEARNED_INSTANCE(8, kFeatAll) KF_LEARNED_INSTANCE(16, 0) KF_LEARNED_INSTANCE(16, kFeatAll)
#undef KF_LEARNED_INSTANCE

}  // namespace kfgb
