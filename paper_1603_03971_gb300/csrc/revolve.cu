// Binomial checkpoint schedules (host code): the dynamic program and the
// action list described in revolve.h.

#include "revolve.h"

#include <map>
#include <memory>
#include <mutex>
#include <utility>

namespace rtm {
namespace {

constexpr double kPlanLimit = 2e9;  // n^2 s inner steps of the dynamic program

struct Plan {
    int n = 0, s = 0;
    std::vector<int64_t> T;  // T[j (n + 1) + m]: j slots, m states
    std::vector<int32_t> C;  // best first advance c for (j, m), j >= 1
    int64_t cost(int j, int m) const { return T[(size_t)j * (n + 1) + m]; }
    int32_t split(int j, int m) const { return C[(size_t)j * (n + 1) + m]; }
};

std::shared_ptr<const Plan> build(int n, int s) {
    auto P = std::make_shared<Plan>();
    P->n = n;
    P->s = s;
    const size_t w = (size_t)n + 1;
    P->T.assign(w * (s + 1), 0);
    P->C.assign(w * (s + 1), 0);
    for (int m = 0; m <= n; m++) P->T[m] = (int64_t)m * (m + 1) / 2;
    for (int j = 1; j <= s; j++) {
        int64_t* Tj = &P->T[(size_t)j * w];
        const int64_t* Tp = &P->T[(size_t)(j - 1) * w];
        int32_t* Cj = &P->C[(size_t)j * w];
        Tj[0] = 0;
        for (int m = 1; m <= n; m++) {
            int64_t best = -1;
            int32_t bc = m;
            for (int c = 1; c <= m; c++) {
                const int64_t v = c + Tp[m - c] + Tj[c - 1];
                if (best < 0 || v < best) {
                    best = v;
                    bc = c;
                }
            }
            Tj[m] = best;
            Cj[m] = bc;
        }
    }
    return P;
}

std::mutex g_mu;
std::map<std::pair<int, int>, std::shared_ptr<const Plan>> g_plans;

std::shared_ptr<const Plan> plan_for(int n, int s) {
    if (n < 0 || s < 0) return nullptr;
    if (s > n) s = n;  // more slots than states do not help
    if ((double)n * n * (s > 0 ? s : 1) > kPlanLimit) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find({n, s});
    if (it != g_plans.end()) return it->second;
    auto P = build(n, s);
    g_plans[{n, s}] = P;
    return P;
}

struct Emitter {
    const Plan& P;
    std::vector<RevolveAction>& out;
    std::vector<int> free_slots;
    int cur = -1;  // state held by the working pair (none known at the start)

    void restore(int slot, int a) {
        if (cur != a) {
            out.push_back({REV_RESTORE, slot, a, 0});
            cur = a;
        }
    }
    // deliver states a + n, ..., a + 1; state a is in `slot` (-1: initial)
    void run(int a, int n, int s, int slot) {
        while (n > 0) {
            if (s == 0) {
                for (int m = n; m >= 1; m--) {
                    restore(slot, a);
                    out.push_back({REV_ADVANCE, a, a + m, 1});
                    cur = a + m;
                    out.push_back({REV_DELIVER, a + m, -1, 0});
                }
                return;
            }
            const int c = P.split(s, n);
            restore(slot, a);
            if (c == n) {
                out.push_back({REV_ADVANCE, a, a + n, 1});
                cur = a + n;
                out.push_back({REV_DELIVER, a + n, -1, 0});
            } else {
                out.push_back({REV_ADVANCE, a, a + c, 0});
                cur = a + c;
                const int sig = free_slots.back();
                free_slots.pop_back();
                out.push_back({REV_STORE, sig, a + c, 0});
                run(a + c, n - c, s - 1, sig);
                out.push_back({REV_DELIVER, a + c, sig, 0});
                out.push_back({REV_FREE, sig, 0, 0});
                free_slots.push_back(sig);
            }
            n = c - 1;  // then the states before the split, from state a again
        }
    }
};

}  // namespace

int64_t revolve_cost(int n, int s) {
    auto P = plan_for(n, s);
    if (!P) return -1;
    return P->cost(P->s, n);
}

bool revolve_schedule(int n, int s, std::vector<RevolveAction>& out) {
    out.clear();
    auto P = plan_for(n, s);
    if (!P) return false;
    Emitter E{*P, out, {}, -1};
    for (int i = P->s - 1; i >= 0; i--) E.free_slots.push_back(i);
    E.run(0, n, P->s, -1);
    return true;
}

}  // namespace rtm
