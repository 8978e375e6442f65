// Dispatch from (w, M, op) to the polynomial-kernel instantiations.  Each
// instantiation is compiled in a translation unit of its own (generated by
// the build from the RSGB_INSTANCE_* macros) so the build runs in parallel.
#include "launch.hpp"

namespace rsgb {

#define RSGB_DECLARE(W, M, OP) \
  cudaError_t launch_poly_w##W##_m##M##_op##OP(const JobParams&, const LaunchShape&, cudaStream_t);
#define RSGB_DECLARE_M(W, OP) \
  RSGB_DECLARE(W, 1, OP) RSGB_DECLARE(W, 2, OP) RSGB_DECLARE(W, 3, OP) RSGB_DECLARE(W, 4, OP) \
  RSGB_DECLARE(W, 5, OP) RSGB_DECLARE(W, 6, OP) RSGB_DECLARE(W, 7, OP) RSGB_DECLARE(W, 8, OP)
RSGB_DECLARE_M(8, 0)
RSGB_DECLARE_M(8, 1)
RSGB_DECLARE_M(16, 0)
RSGB_DECLARE_M(16, 1)

using PolyLauncher = cudaError_t (*)(const JobParams&, const LaunchShape&, cudaStream_t);

#define RSGB_ROW(W, OP)                                                                          \
  {launch_poly_w##W##_m1_op##OP, launch_poly_w##W##_m2_op##OP, launch_poly_w##W##_m3_op##OP,     \
   launch_poly_w##W##_m4_op##OP, launch_poly_w##W##_m5_op##OP, launch_poly_w##W##_m6_op##OP,     \
   launch_poly_w##W##_m7_op##OP, launch_poly_w##W##_m8_op##OP}

static const PolyLauncher kTable[2][2][8] = {
    {RSGB_ROW(8, 0), RSGB_ROW(8, 1)},
    {RSGB_ROW(16, 0), RSGB_ROW(16, 1)},
};

cudaError_t launch_poly(int w, int M, int op, const JobParams& p, const LaunchShape& sh, cudaStream_t st) {
  const int wi = w == 8 ? 0 : (w == 16 ? 1 : -1);
  if (wi < 0 || M < 1 || M > 8 || (op != 0 && op != 1)) return cudaErrorInvalidValue;
  return kTable[wi][op][M - 1](p, sh, st);
}

int poly_max_consumer_warps(int w, int M, int op) {
  return (op == 0 && M * w <= 64) ? 16 : 8;
}

}  // namespace rsgb
