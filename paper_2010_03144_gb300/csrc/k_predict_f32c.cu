// K2 kernels instantiated for float fields in the compact encoding (unpredictable values
// truncated in the full-block walk; see predict.cuh).
#include "predict.cuh"

namespace sdcsz {

void launch_predict_f32_c(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                          const Launch& L) {
  if (g.abft) kpred::launch_predict_t<float, true, true>(field, g, w, flips, nflips, L);
  else kpred::launch_predict_t<float, false, true>(field, g, w, flips, nflips, L);
}

bool batch_predict_fast_f32_c(int ndim, uint32_t B, bool abft, const BatchArgs& a, const Launch& L) {
  return abft ? kpred::batch_fast_shape<float, true, true>(ndim, B, a, L)
              : kpred::batch_fast_shape<float, false, true>(ndim, B, a, L);
}

}  // namespace sdcsz
