// K2 kernels instantiated for float fields (see predict.cuh).
#include "predict.cuh"

namespace sdcsz {

void launch_predict_f32(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                        const Launch& L) {
  if (g.abft) kpred::launch_predict_t<float, true>(field, g, w, flips, nflips, L);
  else kpred::launch_predict_t<float, false>(field, g, w, flips, nflips, L);
}

bool batch_predict_fast_f32(int ndim, uint32_t B, bool abft, const BatchArgs& a, const Launch& L) {
  return abft ? kpred::batch_fast_shape<float, true>(ndim, B, a, L) : kpred::batch_fast_shape<float, false>(ndim, B, a, L);
}

void batch_predict_generic_f32(int ndim, bool abft, const BatchArgs& a, uint32_t threads, size_t smem,
                               const Launch& L) {
  if (abft) kpred::batch_generic_dim<float, true>(ndim, a, threads, smem, L);
  else kpred::batch_generic_dim<float, false>(ndim, a, threads, smem, L);
}

}  // namespace sdcsz
