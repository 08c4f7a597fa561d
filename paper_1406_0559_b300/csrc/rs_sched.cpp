// rs_sched.cpp -- host-only scheduling policy of the map server: which
// queued requests to admit under the device-memory budget, and how many ray
// tiles of each running request go into the next time slice.
//
// Pure functions on plain arrays (no CUDA), so the policy is tested on a
// machine without a GPU.  The paper's survey ran independent map jobs
// through a batch queue (Sec. 2.3); serving requests as they arrive with "a
// scheduler to manage the user requests" is its stated next step (Sec. 5).
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "../../include/rs.h"

extern "C" {

int rs_sched_admit(const rs_sched_queued* q, int n, int64_t bytes_used, int64_t budget,
                   int active, int max_active, int max_skips, int32_t* admit)
{
    if (n < 0 || (n > 0 && (!q || !admit)) || budget < 0 || bytes_used < 0) return RS_EINVAL;
    int admitted = 0;
    for (int k = 0; k < n; ++k) admit[k] = 0;
    for (int k = 0; k < n; ++k) {
        if (active + admitted >= max_active) break;
        if (q[k].bytes > budget) continue;                 // can never fit: caller fails it
        if (bytes_used + q[k].bytes <= budget) {
            admit[k] = 1;
            bytes_used += q[k].bytes;
            ++admitted;
        } else if (q[k].skips >= max_skips) {
            break;   // an old request waits for room: nothing behind it may pass
        }
    }
    return admitted;
}

int rs_sched_plan(const rs_sched_item* items, int n, double budget, int policy, int max_maps,
                  int64_t* take)
{
    if (n < 0 || (n > 0 && (!items || !take)) || max_maps < 1) return RS_EINVAL;
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    for (int k = 0; k < n; ++k) take[k] = 0;
    if (policy == RS_SCHED_SRPT) {
        // shortest remaining work first; ties by arrival
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            const double ra = (double)items[a].tiles_left * items[a].work_per_tile;
            const double rb = (double)items[b].tiles_left * items[b].work_per_tile;
            if (ra != rb) return ra < rb;
            return items[a].seq < items[b].seq;
        });
    } else {
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return items[a].seq < items[b].seq; });
    }
    double left = budget;
    int maps = 0;
    for (int idx : order) {
        const rs_sched_item& it = items[idx];
        if (it.tiles_left <= 0) continue;
        if (maps >= max_maps) break;
        if (left <= 0.0 && maps > 0) break;
        int64_t k = it.tiles_left;
        if (it.work_per_tile > 0.0 && isfinite(budget)) {
            const double fit = floor(left / it.work_per_tile);
            if (fit < (double)k) k = fit < 1.0 ? 1 : (int64_t)fit;   // always progress
        }
        take[idx] = k;
        left -= (double)k * it.work_per_tile;
        ++maps;
    }
    return maps;
}

}  // extern "C"
