// Instances of the fused direct-forcing kernel for blocks of 256 threads (a
// translation unit of its own, so that the two block sizes compile in
// parallel).
#include "force_tile.cuh"

namespace mls {

const void* force_kernel_256(bool bf, bool vec, int lx, int ly, int lz) {
  constexpr int NT = kForceThreads;
  return bf ? (vec ? force_kernel<__nv_bfloat16, true, NT>(lx, ly, lz) : force_kernel<__nv_bfloat16, false, NT>(lx, ly, lz))
            : (vec ? force_kernel<float, true, NT>(lx, ly, lz) : force_kernel<float, false, NT>(lx, ly, lz));
}

}  // namespace mls
