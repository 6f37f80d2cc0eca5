// K2 kernels instantiated for double fields in the raw encoding (see predict.cuh); the compact
// encoding's full-block kernels are instantiated in k_predict_f64c.cu.
#include "predict.cuh"

namespace sdcsz {

void launch_predict_f64_c(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                          const Launch& L);
bool batch_predict_fast_f64_c(int ndim, uint32_t B, bool abft, const BatchArgs& a, const Launch& L);

void launch_predict_f64(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                        const Launch& L) {
  if (g.enc) launch_predict_f64_c(field, g, w, flips, nflips, L);
  else if (g.abft) kpred::launch_predict_t<double, true, false>(field, g, w, flips, nflips, L);
  else kpred::launch_predict_t<double, false, false>(field, g, w, flips, nflips, L);
}

bool batch_predict_fast_f64(int ndim, uint32_t B, bool abft, bool enc, const BatchArgs& a, const Launch& L) {
  if (enc) return batch_predict_fast_f64_c(ndim, B, abft, a, L);
  return abft ? kpred::batch_fast_shape<double, true, false>(ndim, B, a, L)
              : kpred::batch_fast_shape<double, false, false>(ndim, B, a, L);
}

void batch_predict_generic_f64(int ndim, bool abft, const BatchArgs& a, uint32_t threads, size_t smem,
                               const Launch& L) {
  if (abft) kpred::batch_generic_dim<double, true>(ndim, a, threads, smem, L);
  else kpred::batch_generic_dim<double, false>(ndim, a, threads, smem, L);
}

}  // namespace sdcsz
