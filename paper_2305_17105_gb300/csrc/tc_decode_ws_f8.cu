// FP8-E4M3 form of the warp-specialised tensor-core decode (kind::f8f6f4),
// one instantiation per fast-layout class and the generic layout; its own
// translation unit so that it compiles beside the FP16 instantiations.
#include "tc_decode_ws.cuh"

namespace ntc {

cudaError_t launch_decode_ws_f8(const ntc_material& m, const float* uvl, int64_t n, void* out,
                                int out_dtype, int filter, uint64_t jkey, cudaStream_t s) {
  const Plan P(m, true, fast_layout_ok(m));
  if (!P.fast) return launch_ws<0, true>(m, uvl, n, out, out_dtype, filter, jkey, s);
  switch (1 + 3 * grid_class(m.c0, P.cb0) + grid_class(m.c1, P.cb1)) {
    case 1: return launch_ws<1, true>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 2: return launch_ws<2, true>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 3: return launch_ws<3, true>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 4: return launch_ws<4, true>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 5: return launch_ws<5, true>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 6: return launch_ws<6, true>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 7: return launch_ws<7, true>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 8: return launch_ws<8, true>(m, uvl, n, out, out_dtype, filter, jkey, s);
    default: return launch_ws<9, true>(m, uvl, n, out, out_dtype, filter, jkey, s);
  }
}

}  // namespace ntc
