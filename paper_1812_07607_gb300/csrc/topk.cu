// topk.cu -- top-k join (Sec. 6.2 q1: nearest image to a query image, generalised to k).
#include "kernels.h"

using namespace dl;

extern "C" int dl_topk_join(const dl_store *Q, const dl_store *S, int32_t metric, int32_t k, const dl_join_opts *opts,
                            dl_result **out)
{
    clear_error();
    (void)Q;
    (void)S;
    (void)metric;
    (void)k;
    (void)opts;
    if (out) *out = nullptr;
    set_error("dl_topk_join: not available in this build yet");
    return DL_EUNSUPPORTED;
}
