// Device side of the persistent wavefront schedule (shared by the persistent kernels): product
// claims from a counter, acquire / release completion flags, and bounded waits for the products
// a product reads.
#pragma once
#include "kernels.h"

__device__ __forceinline__ unsigned long long f2_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int wave_claim(const WaveArgs& A) {
    if (*reinterpret_cast<volatile int*>(&A.ctl->abort)) return A.ntask;
    return atomicAdd(&A.ctl->next, 1);
}

// Warp 0 waits: lane q polls the flags of dependencies q, q + 32, ... (one round trip to L2 for
// all of them instead of one per dependency), each lane bounded by wait_ns.
__device__ __forceinline__ void wave_wait_warp(const WaveArgs& A, int i, int epoch, int lane) {
    const int d0 = A.tasks[i].dep0, nd = A.tasks[i].ndep;
    unsigned long long t0 = 0;
    for (int q = lane; q < nd; q += 32) {
        const int* f = A.flags + A.deps[d0 + q];
        while (ld_acquire_gpu(f) != epoch) {
            if (*reinterpret_cast<volatile int*>(&A.ctl->abort)) return;
            const unsigned long long now = f2_globaltimer();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > A.wait_ns) {
                atomicOr(A.err, 4);
                atomicExch(&A.ctl->abort, 1);
                return;
            }
            __nanosleep(32);
        }
    }
}
