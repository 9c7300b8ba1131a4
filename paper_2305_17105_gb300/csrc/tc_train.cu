// Launchers of the fused training step (one material per launch), the
// kernel itself lives in tc_train.cuh.
#include "tc_train.cuh"

namespace ntc {

bool train_tc_supported(const ntc_material& m) {
  if (m.act != NTC_ACT_RELU && m.act != NTC_ACT_HARDGELU) return false;
  if (m.precision == NTC_PREC_F8)  // FP8 form: bilinear G0, two hidden layers, K in 32s
    return m.interp0 == NTC_INTERP_BILINEAR && m.hidden_layers != 3 && m.k_in % 32 == 0 &&
           m.vq_books == 0 && m.scale != nullptr && train_pipelines(m) > 0;
  return m.precision == NTC_PREC_F16 && train_pipelines(m) > 0;
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
  if (m.precision == NTC_PREC_F8) return launch_train_tc_f8(m, a, s);
  return launch_class<false>(m, a, nullptr, (a.n + kRows - 1) / kRows, 0, 0, s);
}


}  // namespace ntc
