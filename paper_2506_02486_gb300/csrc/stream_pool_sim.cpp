// stream_pool_sim.cpp -- gw_stream_pool_simulate: the stream pool's policy
// (stream_pool.h) driven by a host-side model with a logical clock, so the
// policy can be tested without a GPU and the threshold sized offline.
#include <algorithm>
#include <vector>

#include "gw_internal.h"

namespace gw {
namespace {

// A stream is an index; it is idle once the clock has passed the completion
// tick of its last operation.  Waiting moves the clock forward.
struct SimStreams {
    using Handle = int;
    long long *clock = nullptr;
    std::vector<long long> *done_at = nullptr;
    gw_status create(Handle *h)
    {
        *h = (int)done_at->size();
        done_at->push_back(0);
        return GW_OK;
    }
    gw_status done(Handle h, bool *d)
    {
        *d = (*done_at)[h] <= *clock;
        return GW_OK;
    }
    gw_status sync(Handle h)
    {
        *clock = std::max(*clock, (*done_at)[h]);
        return GW_OK;
    }
    void destroy(Handle) {}
};

}  // namespace
}  // namespace gw

using namespace gw;

extern "C" gw_status gw_stream_pool_simulate(int max_active, int nops,
                                             const int *duration, int *stream_of_op,
                                             gw_pool_stats *out)
{
    if (max_active < 1 || max_active > 64)
        return fail(GW_ERR_ARG, "max active streams must be 1 .. 64, got %d", max_active);
    if (nops < 0 || (nops > 0 && !duration) || !out) return fail(GW_ERR_ARG, "bad arguments");
    for (int i = 0; i < nops; ++i)
        if (duration[i] < 0) return fail(GW_ERR_ARG, "duration[%d] < 0", i);
    long long clock = 0;
    std::vector<long long> done_at;
    SimStreams be;
    be.clock = &clock;
    be.done_at = &done_at;
    StreamPool<SimStreams> pool(be);
    pool.set_max_active(max_active);
    for (int i = 0; i < nops; ++i) {
        int idx = -1;
        GW_TRY(pool.acquire(&idx));
        const int h = pool.handle(idx);
        done_at[h] = std::max(done_at[h], clock) + duration[i];
        if (stream_of_op) stream_of_op[i] = idx;
        ++clock;
    }
    *out = pool.stats();
    return GW_OK;
}
