// K2 kernels instantiated for double fields (see predict.cuh).
#include "predict.cuh"

namespace sdcsz {

void launch_predict_f64(const void* field, const Geo& g, const Ws& w, const sdcsz_flip* flips, uint32_t nflips,
                        const Launch& L) {
  if (g.abft) kpred::launch_predict_t<double, true>(field, g, w, flips, nflips, L);
  else kpred::launch_predict_t<double, false>(field, g, w, flips, nflips, L);
}

}  // namespace sdcsz
