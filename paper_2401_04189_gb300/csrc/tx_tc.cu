// Tensor-core (tcgen05 / TMEM / TMA) path.
#include <cuda_runtime.h>

#include <string>

#include "tx_paths.h"

namespace tx {

bool tc_supported(const tx_ctx* c, std::string* why) {
    (void)c;
    if (why) *why = "tensor-core precisions are not built yet";
    return false;
}
int tc_prepare(tx_ctx* c, cudaStream_t s) {
    (void)c;
    (void)s;
    return fail(TX_ERR_UNSUPPORTED_PRECISION, "tensor-core precisions are not built yet");
}
void tc_release(tx_ctx* c) { (void)c; }
size_t tc_batch_bytes_per_pair(const tx_ctx* c, int kind) {
    (void)c;
    (void)kind;
    return 0;
}
long tc_epart_per_pair(const tx_ctx* c) {
    (void)c;
    return 0;
}
int tc_run_batch(tx_ctx* c, const CallSpec& cs, const BatchBuffers& b, cudaStream_t s) {
    (void)c;
    (void)cs;
    (void)b;
    (void)s;
    return fail(TX_ERR_UNSUPPORTED_PRECISION, "tensor-core precisions are not built yet");
}

}  // namespace tx
