// Binomial checkpoint schedules for the reverse sweep of the imaging pass
// (host code).
//
// The receiver pass needs the source wavefield at the imaging steps in
// reverse order. Coarse state X_j is the leapfrog pair (u^{j k - 1}, u^{j k})
// of imaging step j k (k = image_every); X_0 is the zero initial state and is
// always available. With s checkpoint slots, the fewest coarse forward steps
// T(n, s) that deliver X_n, X_{n-1}, ..., X_1 in that order, starting from
// X_0, obey
//   T(0, s) = 0,   T(n, 0) = n (n + 1) / 2   (every state from X_0 again),
//   T(n, s) = min_{1 <= c <= n} [ c + T(n - c, s - 1) + T(c - 1, s) ]
// (advance c steps; if c < n keep X_c in a slot, deliver the n - c later
// states with one slot fewer, deliver X_c from its slot and free it; then
// the c - 1 earlier states from X_0 again), the recursion behind binomial
// (revolve) checkpointing. Table and split points are computed once per
// (n, s) by dynamic programming, O(n^2 s). The schedule assumes nothing
// about the working pair at its start: its first action restores X_0.
#pragma once

#include <stdint.h>

#include <vector>

namespace rtm {

enum RevolveOp : int32_t {
    REV_RESTORE = 0,  // a = slot (-1: the zero initial state), b = state restored
    REV_ADVANCE = 1,  // from state a to state b; c = 1: write the imaging snapshot at the end
    REV_STORE = 2,    // a = slot, b = state stored (the working pair)
    REV_DELIVER = 3,  // a = state; b = -1: the working pair and the snapshot just written,
                      // b >= 0: the slot that holds it
    REV_FREE = 4,     // a = slot
};

struct RevolveAction {
    int32_t op, a, b, c;
};

// minimal coarse forward steps (-1 if n * n * s exceeds the planning limit)
int64_t revolve_cost(int n, int s);
// the schedule; false if over the planning limit
bool revolve_schedule(int n, int s, std::vector<RevolveAction>& out);

}  // namespace rtm
