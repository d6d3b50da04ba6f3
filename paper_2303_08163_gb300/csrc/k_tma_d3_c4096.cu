// k_tma_d3_c4096.cu -- TMA row-staged step kernels for D = 3, 4096-byte direction buffers.
#include "k_tma.cuh"

namespace lbmh {
const void *tma_kernel_d3_c4096(int P, int eq, int bulk) { return lbmd::tma_kernel_dc<3, 4096>(P, eq, bulk); }
}  // namespace lbmh
