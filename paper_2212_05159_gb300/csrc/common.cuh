// Shared helpers of the CUDA sources: status handling, launch checks, warp utilities.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/spx.h"

namespace spx {

// Records a message for spx_last_error() (thread-local) and returns the status.
spx_status set_error(spx_status st, const char* fmt, ...);

// Translates a CUDA runtime error into SPX_CUDA_ERROR with a message.
spx_status cuda_error(cudaError_t err, const char* where);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

constexpr unsigned FULL = 0xffffffffu;
constexpr int NUM_SMS_GB300 = 152;

// Number of SMs of the current device (cached per process; GB300 has 152).
int num_sms();

// Checks the header of a CSR view (not its contents).
spx_status check_csr(const spx_csr* A, bool need_values, const char* who);

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// L2 eviction-priority policies (PTX createpolicy): CSR index / value streams are read
// once and marked evict-first; the gathered dense slab is marked evict-last so that it
// stays resident while the streams pass through.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ int ld_hint(const int* p, uint64_t pol) {
    int v;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float ld_hint(const float* p, uint64_t pol) {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
// 16-byte gathers of dense rows through a column stream: not kept in L1 (their reuse is in
// L2, if anywhere; measured 1 % faster on the power-law SpMM, equal elsewhere)
__device__ __forceinline__ float4 ld_hint4(const float* p, uint64_t pol) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p), "l"(pol));
    return v;
}

// ---- TMA-engine bulk copies and mbarriers (sm_90+ PTX) ---------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// global -> shared copy by the TMA engine; completion counted on the mbarrier in bytes.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// orders this thread's earlier generic-proxy shared-memory accesses before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for the phase with the given parity to complete, giving up after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// Device address of the library's error word (bit 0: a bounded device-side wait ran out),
// for kernels to record failures in; read and cleared by spx_check_device().
int* device_error_word();

// Streaming loads for data read exactly once (evict-first).
__device__ __forceinline__ int ld_stream(const int* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }

}  // namespace spx

#define SPX_CHECK_LAUNCH(where)                                        \
    do {                                                               \
        cudaError_t e_ = cudaGetLastError();                           \
        if (e_ != cudaSuccess) return ::spx::cuda_error(e_, where);    \
    } while (0)

#define SPX_CUDA(call, where)                                          \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return ::spx::cuda_error(e_, where);    \
    } while (0)

#define SPX_TRY(call)                                                  \
    do {                                                               \
        spx_status s_ = (call);                                        \
        if (s_ != SPX_OK) return s_;                                   \
    } while (0)

namespace spx {

// Raises the dynamic shared-memory limit of `kern` to `bytes` once per device (the attribute
// belongs to the device's context); `done` holds one bit per device id below 64 and makes
// concurrent first calls from several threads harmless (the attribute call is idempotent).
template <typename K>
inline spx_status ensure_smem_attr(K kern, int bytes, std::atomic<unsigned long long>& done, const char* who) {
    int dev = 0;
    SPX_CUDA(cudaGetDevice(&dev), who);
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return SPX_OK;
    SPX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes), who);
    if (bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return SPX_OK;
}

}  // namespace spx
