// The screening launches with the query tiles in tensor memory (d_pad = 128,
// no exclusion radius), with the bound check compiled out or in.
#include "tc_scan_kernel.cuh"

namespace osann {

int launch_tc_scan_tmem(const void* maps, const TcArgs& a, int k, int prec, bool debug, cudaStream_t st, int num_sms)
{
    if (a.d_pad != 128) return -2;
#define OSANN_TC(KM)                                                                                 \
    do {                                                                                             \
        if (debug)                                                                                   \
            return prec == 0 ? launch_tc_t<KM, false, 0, true, true>(maps, a, st, num_sms)           \
                             : launch_tc_t<KM, false, 1, true, true>(maps, a, st, num_sms);          \
        return prec == 0 ? launch_tc_t<KM, false, 0, false, true>(maps, a, st, num_sms)              \
                         : launch_tc_t<KM, false, 1, false, true>(maps, a, st, num_sms);             \
    } while (0)
    if (k <= 1) OSANN_TC(1);
    if (k <= 4) OSANN_TC(4);
    if (k <= 16) OSANN_TC(16);
    OSANN_TC(32);
#undef OSANN_TC
}

}  // namespace osann
