// k_tma_d2_c1024.cu -- TMA row-staged step kernels for D = 2, 1024-byte direction buffers.
#include "k_tma.cuh"

namespace lbmh {
const void *tma_kernel_d2_c1024(int P, int eq, int bulk) { return lbmd::tma_kernel_dc<2, 1024>(P, eq, bulk); }
}  // namespace lbmh
