// The screening launch with the bound check compiled in (OSANN_DEBUG_CHECKS=1):
// every screened value is compared with an fp32 evaluation of the folded
// product, and a violation sets OSANN_STATUS_BOUND.
#include "tc_scan_kernel.cuh"

namespace osann {

int launch_tc_scan_debug(const void* maps, const TcArgs& a, int k, int prec, bool excl, cudaStream_t st, int num_sms)
{
#define OSANN_TC(KM)                                                                                 \
    do {                                                                                             \
        if (prec == 0)                                                                               \
            return excl ? launch_tc_t<KM, true, 0, true>(maps, a, st, num_sms)                       \
                        : launch_tc_t<KM, false, 0, true>(maps, a, st, num_sms);                     \
        return excl ? launch_tc_t<KM, true, 1, true>(maps, a, st, num_sms)                           \
                    : launch_tc_t<KM, false, 1, true>(maps, a, st, num_sms);                         \
    } while (0)
    if (k <= 1) OSANN_TC(1);
    if (k <= 4) OSANN_TC(4);
    if (k <= 16) OSANN_TC(16);
    OSANN_TC(32);
#undef OSANN_TC
}

}  // namespace osann
