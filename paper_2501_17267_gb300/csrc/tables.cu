// tables.cu -- beta schedules and integer acceptance thresholds (host).
//
// Every accept decision on the device is an integer compare of a 32-bit Philox
// word u against a threshold computed here once, in IEEE double with the C
// library's exp:  accept an energy increase dE when u < floor(2^32 exp(-beta dE)),
// clamped to 2^32 - 1.  No transcendental function runs on the device.
//
// Schedules: App. D.1 anneals along a geometric beta schedule; linear schedules are
// supported too.  App. D.2 uses a geometric ladder for parallel tempering.  One
// sweep per schedule value; the last value is the end point exactly.
#include <math.h>

#include "sg_internal.h"

namespace sg {

void beta_schedule(int S, double b0, double b1, int geometric, double* beta)
{
    for (int s = 0; s < S; ++s) {
        double v;
        if (S == 1)
            v = b0;
        else if (s == S - 1)
            v = b1;
        else if (geometric)
            v = b0 * pow(b1 / b0, (double)s / (double)(S - 1));
        else
            v = b0 + (b1 - b0) * (double)s / (double)(S - 1);
        beta[s] = v;
    }
}

static uint32_t threshold(double rate, double gap)
{
    const double v = floor(ldexp(exp(-(rate * gap)), 32));
    return v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
}

void metropolis_row(double beta, uint32_t* row)
{
    row[0] = 0xFFFFFFFFu;  // dE = 0 is always accepted by the kernel; entry unused
    for (int k = 1; k < kThrRow; ++k) row[k] = k <= kMaxK ? threshold(beta, (double)(2 * k)) : 0u;
}

uint32_t exchange_threshold(double dbeta, int64_t d) { return threshold(dbeta, (double)d); }

int32_t build_exchange_tables(const std::vector<double>& ladder, int64_t dmax, ExchangeTables* out)
{
    const int K = (int)ladder.size();
    out->tab.clear();
    out->off.assign(K > 1 ? K - 1 : 1, 0);
    out->len.assign(K > 1 ? K - 1 : 1, 0);
    out->tail.assign(K > 1 ? K - 1 : 1, 0);
    constexpr int64_t kCap = int64_t(1) << 22;
    for (int k = 0; k + 1 < K; ++k) {
        const double db = ladder[k + 1] - ladder[k];
        out->off[k] = (uint32_t)out->tab.size();
        if (!(db > 0)) {
            // equal (or decreasing) rungs: exp(-db d) >= 1 for every d >= 1, so every
            // positive gap gives the clamp value
            out->len[k] = 0;
            out->tail[k] = 0xFFFFFFFFu;
            continue;
        }
        int64_t d = 1;
        for (; d <= dmax; ++d) {
            const uint32_t t = threshold(db, (double)d);
            if (t == 0) break;
            if (d > kCap) {
                set_error("PT ladder spacing %.3g is too fine: exchange table exceeds %lld entries",
                          db, (long long)kCap);
                return SG_EINVAL;
            }
            out->tab.push_back(t);
        }
        out->len[k] = (uint32_t)(d - 1);
        out->tail[k] = 0;  // exp(-db d) only decreases beyond the first zero
    }
    if (out->tab.empty()) out->tab.push_back(0);
    return SG_OK;
}

}  // namespace sg
