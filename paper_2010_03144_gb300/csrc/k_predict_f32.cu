// K2 kernels instantiated for float fields (see predict.cuh).
#include "predict.cuh"

namespace sdcsz {

void launch_predict_f32(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                        const Launch& L) {
  if (g.abft) kpred::launch_predict_t<float, true>(field, g, w, flips, nflips, L);
  else kpred::launch_predict_t<float, false>(field, g, w, flips, nflips, L);
}

}  // namespace sdcsz
