// TT rounding, sparse TT-SVD compression and the QTT inverse.
#include "internal.cuh"

extern "C" {
int qtt_round(qp_ctx_t, qtt_t, double, int, qtt_t*) { return QP_NOT_READY; }
int qtt_compress(qp_ctx_t, const qp_state*, double, int, qtt_t*) { return QP_NOT_READY; }
int qtt_inverse(qp_ctx_t, qtt_t, double, int, int, qtt_t, qtt_t*) { return QP_NOT_READY; }
}
