// k_tma_d3_c8192.cu -- TMA row-staged step kernels for D = 3, 8192-byte direction buffers.
#include "k_tma.cuh"

namespace lbmh {
const void *tma_kernel_d3_c8192(int P, int eq, int bulk) { return lbmd::tma_kernel_dc<3, 8192>(P, eq, bulk); }
}  // namespace lbmh
