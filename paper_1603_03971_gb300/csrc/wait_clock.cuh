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

// one poll of an mbarrier phase (shared-memory address a) that lets the
// thread sleep until the phase completes or suspend_ns nanoseconds pass:
// a thread that waits long stays off the issue slots and the shared-memory
// pipe instead of re-polling
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t a, uint32_t parity,
                                                    uint32_t suspend_ns) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(suspend_ns)
        : "memory");
    return done != 0;
}

}  // namespace rtm
