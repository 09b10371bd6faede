// stream_pool.h -- the bounded stream pool behind the non-blocking puts and
// gets (paper section 3.2, "Bounded Concurrency").
//
// Streams are created lazily, one per concurrent operation, and reused once
// released.  At most `max_active` streams carry operations that have not been
// released.  When an operation needs a stream and that many are active, the
// pool synchronises part of them: it queries the active streams, and of those
// whose work has completed it releases half (rounded up, oldest activation
// first); the other active streams keep running.  When none has completed it
// waits for the oldest active stream and releases that one.  A fence releases
// every active stream after joining it into the fence's stream.
//
// The policy is written against a backend (create / done / sync / destroy of
// an opaque stream handle) so the same code runs on CUDA streams and on a
// host-side simulation with a logical clock.
#pragma once
#include <algorithm>
#include <cstdint>
#include <vector>

#include "gbwave.h"

namespace gw {

#define GW_POOL_TRY(call)                \
    do {                                 \
        gw_status s_ = (call);           \
        if (s_ != GW_OK) return s_;      \
    } while (0)

template <class Backend>
class StreamPool {
public:
    using Handle = typename Backend::Handle;

    explicit StreamPool(Backend be = Backend()) : be_(be) {}
    StreamPool(const StreamPool &) = delete;
    StreamPool &operator=(const StreamPool &) = delete;

    Backend &backend() { return be_; }
    int max_active() const { return max_active_; }
    void set_max_active(int n) { max_active_ = n; }

    // A stream for one new operation, marked active.  *idx: its index.
    gw_status acquire(int *idx)
    {
        if ((int)active_.size() >= max_active_) GW_POOL_TRY(partial_sync());
        int s;
        if (!idle_.empty()) {
            s = idle_.front();
            idle_.erase(idle_.begin());
            ++st_.reuses;
        } else {
            Handle h{};
            GW_POOL_TRY(be_.create(&h));
            streams_.push_back(h);
            s = (int)streams_.size() - 1;
            ++st_.created;
        }
        active_.push_back(s);            // in activation order
        ++st_.ops;
        st_.peak_active = std::max(st_.peak_active, (int)active_.size());
        *idx = s;
        return GW_OK;
    }

    Handle handle(int idx) const { return streams_[idx]; }

    // Active streams, oldest activation first (for fences).
    const std::vector<int> &active() const { return active_; }

    // Release every active stream (after the caller joined or synced them).
    void release_all()
    {
        for (int s : active_) idle_.push_back(s);
        active_.clear();
    }

    // Host wait for every active stream, then release them.
    gw_status quiet()
    {
        for (int s : active_) GW_POOL_TRY(be_.sync(streams_[s]));
        release_all();
        return GW_OK;
    }

    void destroy()
    {
        for (Handle h : streams_) be_.destroy(h);
        streams_.clear();
        active_.clear();
        idle_.clear();
    }

    gw_pool_stats stats() const
    {
        gw_pool_stats s = st_;
        s.active = (int)active_.size();
        s.idle = (int)idle_.size();
        s.max_active = max_active_;
        return s;
    }

    void count_fence() { ++st_.fences; }

private:
    gw_status partial_sync()
    {
        ++st_.partial_syncs;
        std::vector<int> done;
        for (int s : active_) {
            bool d = false;
            GW_POOL_TRY(be_.done(streams_[s], &d));
            if (d) done.push_back(s);
        }
        std::vector<int> rel;
        if (done.empty()) {
            // nothing has finished: wait for the oldest operation
            const int s = active_.front();
            GW_POOL_TRY(be_.sync(streams_[s]));
            rel.push_back(s);
            ++st_.waited_oldest;
        } else {
            const size_t k = (done.size() + 1) / 2;
            for (size_t i = 0; i < k; ++i) {
                GW_POOL_TRY(be_.sync(streams_[done[i]]));   // returns at once
                rel.push_back(done[i]);
            }
        }
        // release the chosen streams (idle queue in release order) while
        // keeping the others in activation order
        std::vector<int> keep;
        for (int s : active_)
            if (std::find(rel.begin(), rel.end(), s) == rel.end()) keep.push_back(s);
        active_.swap(keep);
        for (int s : rel) idle_.push_back(s);
        st_.released += (long long)rel.size();
        // a lowered limit is honoured by releasing more of the oldest
        while ((int)active_.size() >= max_active_ && !active_.empty()) {
            const int s = active_.front();
            GW_POOL_TRY(be_.sync(streams_[s]));
            active_.erase(active_.begin());
            idle_.push_back(s);
            ++st_.released;
            ++st_.waited_oldest;
        }
        return GW_OK;
    }

    Backend be_;
    int max_active_ = 8;
    std::vector<Handle> streams_;
    std::vector<int> active_;   // indices, oldest activation first
    std::vector<int> idle_;     // indices, reuse order (first released first)
    gw_pool_stats st_{};
};

#undef GW_POOL_TRY

}  // namespace gw
