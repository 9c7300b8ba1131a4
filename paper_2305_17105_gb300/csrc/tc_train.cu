// Launchers of the fused training step (one material per launch), the
// kernel itself lives in tc_train.cuh.
#include "tc_train.cuh"

namespace ntc {

bool train_tc_supported(const ntc_material& m) {
  return m.precision == NTC_PREC_F16 && (m.act == NTC_ACT_RELU || m.act == NTC_ACT_HARDGELU) &&
         train_pipelines(m) > 0;
}

void train_widths(const ntc_material& m, int* k_int, int* dx_n) {
  const TPlan P(m.c0, m.c1, m.interp0 == NTC_INTERP_LEARNED, m.act == NTC_ACT_HARDGELU, 1,
                m.hidden_layers == 3);
  *k_int = P.k_int;
  *dx_n = P.dx_n;
}

int train_pipelines_layout(const ntc_material& first, int k_lay, int dx_lay) {
  return pipelines_for(first, k_lay, dx_lay);
}

cudaError_t launch_train_tc(const ntc_material& m, const BwdArgs& a, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (!train_tc_supported(m) || (!a.train && !a.dout)) return cudaErrorNotSupported;
  return launch_class<false>(m, a, nullptr, (a.n + kRows - 1) / kRows, 0, 0, s);
}


}  // namespace ntc
