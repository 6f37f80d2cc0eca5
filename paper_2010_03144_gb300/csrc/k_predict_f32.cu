// K2 kernels instantiated for float fields in the raw encoding (see predict.cuh); the compact
// encoding's full-block kernels are instantiated in k_predict_f32c.cu.
#include "predict.cuh"

namespace sdcsz {

void launch_predict_f32_c(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                          const Launch& L);
bool batch_predict_fast_f32_c(int ndim, uint32_t B, bool abft, const BatchArgs& a, const Launch& L);

void launch_predict_f32(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                        const Launch& L) {
  if (g.enc) launch_predict_f32_c(field, g, w, flips, nflips, L);
  else if (g.abft) kpred::launch_predict_t<float, true, false>(field, g, w, flips, nflips, L);
  else kpred::launch_predict_t<float, false, false>(field, g, w, flips, nflips, L);
}

bool batch_predict_fast_f32(int ndim, uint32_t B, bool abft, bool enc, const BatchArgs& a, const Launch& L) {
  if (enc) return batch_predict_fast_f32_c(ndim, B, abft, a, L);
  return abft ? kpred::batch_fast_shape<float, true, false>(ndim, B, a, L)
              : kpred::batch_fast_shape<float, false, false>(ndim, B, a, L);
}

void batch_predict_generic_f32(int ndim, bool abft, const BatchArgs& a, uint32_t threads, size_t smem,
                               const Launch& L) {
  if (abft) kpred::batch_generic_dim<float, true>(ndim, a, threads, smem, L);
  else kpred::batch_generic_dim<float, false>(ndim, a, threads, smem, L);
}

}  // namespace sdcsz
