// Pieces shared by the tensor-core stage kernels (net_bf16.cu, net_fp8.cu):
// tile geometry, shared-memory and cp.async helpers, bounded mbarrier waits,
// BF16 chunk conversions and the ring-slot arithmetic of the staged rows.
#pragma once

#include <cstdint>

#include "tc_common.cuh"

namespace nsm {
using namespace tc;

constexpr int kTileM = 128;      // pixels per MMA row block
constexpr int kSW = 136;         // staged pixels per row (128 + halo + pad)
constexpr int kNCC = 66;         // coarse-level columns behind one tile
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s bound on every mbarrier wait

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" :: "r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ uint4 ld_shared_v4(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr)
                 : "memory");
    return v;
}
__device__ __forceinline__ float4 ld_shared_f4(uint32_t addr) {
    const uint4 u = ld_shared_v4(addr);
    return make_float4(__uint_as_float(u.x), __uint_as_float(u.y), __uint_as_float(u.z), __uint_as_float(u.w));
}
// 16-byte asynchronous copy global -> shared; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(saddr), "l"(src), "r"(src_bytes) : "memory");
}
// arrive on mbar once every cp.async this thread issued so far has landed
__device__ __forceinline__ void cp_async_arrive(uint64_t* mbar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" :: "r"(smem_u32(mbar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" :: "r"(smem_u32(mbar))
                 : "memory");
}
// Bounded wait that also gives up when another role of the CTA has aborted.
__device__ __forceinline__ bool wait_phase(uint64_t* mbar, uint32_t parity, const volatile int* abort_flag) {
    if (mbar_try_wait(mbar, parity)) return true;
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        __nanosleep(64);
        if (mbar_try_wait(mbar, parity)) return true;
        if (*abort_flag) return false;
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > kWaitNs) return false;
    }
    return false;
}

// 8 BF16 values of a chunk -> FP32
__device__ __forceinline__ void chunk_to_f32(uint4 c, float (&f)[8]) {
    float2 a = unpack_bf16x2(c.x), b = unpack_bf16x2(c.y), d = unpack_bf16x2(c.z), e = unpack_bf16x2(c.w);
    f[0] = a.x; f[1] = a.y; f[2] = b.x; f[3] = b.y; f[4] = d.x; f[5] = d.y; f[6] = e.x; f[7] = e.y;
}
__device__ __forceinline__ uint4 f32_to_chunk(const float* f) {
    return make_uint4(pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]), pack_bf16x2(f[4], f[5]),
                      pack_bf16x2(f[6], f[7]));
}

// staged row sr of a tile lives in row slot (base + sr) mod NRW of every plane
template <int NRW>
__device__ __forceinline__ int row_slot(int base, int sr) {
    const int q = base + sr;
    return q >= NRW ? q - NRW : q;
}

}  // namespace nsm
