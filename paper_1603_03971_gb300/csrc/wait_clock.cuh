// Time bound of the device spin waits.
//
// Every poll loop on an mbarrier also gives up once kWaitNs nanoseconds of
// %globaltimer time have passed since it began. A try_wait may suspend the
// thread for an implementation-defined time on each poll, so a poll count
// alone does not bound how long a wait lasts; the counts stay as a backstop.
#pragma once

namespace rtm {

constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long wait_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// true once a wait that began at t0 has run out of time (read every 256 polls)
__device__ __forceinline__ bool wait_expired(long long poll, unsigned long long t0) {
    return (poll & 255) == 255 && wait_now() - t0 > kWaitNs;
}

}  // namespace rtm
