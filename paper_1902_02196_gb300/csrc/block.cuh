// Constant tables of the 12 x 12 Green block and cp.async helpers shared by the matvec kernels.
#pragma once

#include "common.cuh"

// ---------------------------------------------------------------------------
// Constant table: for each unique tensor t the (alpha, beta, sign) entries of the 12x12 block
// ---------------------------------------------------------------------------
struct BlockEntry {
    signed char a, b, s;
};
struct BlockTable {
    BlockEntry e[144];
    int start[61];
};
constexpr BlockTable make_block_table() {
    BlockTable T{};
    int n = 0;
    for (int t = 0; t < 60; ++t) {
        T.start[t] = n;
        for (int a = 0; a < 12; ++a)
            for (int b = 0; b < 12; ++b)
                if (tensor_of(a, b) == t) {
                    T.e[n].a = (signed char)a;
                    T.e[n].b = (signed char)b;
                    T.e[n].s = (signed char)sign_of(a, b);
                    ++n;
                }
    }
    T.start[60] = n;
    return T;
}
__device__ constexpr BlockTable kBlock = make_block_table();
static_assert(make_block_table().start[60] == 144, "every block entry maps to one of the 60 tensors");

// The same 144 entries ordered by input component b, then output a: consecutive
// multiply-adds go to different accumulators, so each accumulator's chain of dependent
// FMAs is interleaved with the other rows' (FMA latency hidden within one thread).
struct BlockEntryT {
    signed char a, b, t, s;
};
struct BlockTableB {
    BlockEntryT e[144];
};
constexpr BlockTableB make_block_table_b() {
    BlockTableB T{};
    int n = 0;
    for (int b = 0; b < 12; ++b)
        for (int a = 0; a < 12; ++a) {
            T.e[n].a = (signed char)a;
            T.e[n].b = (signed char)b;
            T.e[n].t = (signed char)tensor_of(a, b);
            T.e[n].s = (signed char)sign_of(a, b);
            ++n;
        }
    return T;
}
__device__ constexpr BlockTableB kBlockB = make_block_table_b();

// The 96 non-zero entries of the K block (kblock.h) grouped by the 30 stored tensors
#include "kblock.h"
struct KBlockTable {
    BlockEntry e[96];
    int start[31];
};
constexpr KBlockTable make_kblock_table() {
    KBlockTable T{};
    int n = 0;
    for (int t = 0; t < 30; ++t) {
        T.start[t] = n;
        for (int a = 0; a < 12; ++a)
            for (int b = 0; b < 12; ++b)
                if (kblock::tensor(a, b) == t) {
                    T.e[n].a = (signed char)a;
                    T.e[n].b = (signed char)b;
                    T.e[n].s = (signed char)kblock::sign(a, b);
                    ++n;
                }
    }
    T.start[30] = n;
    return T;
}
__device__ constexpr KBlockTable kKBlock = make_kblock_table();
static_assert(make_kblock_table().start[30] == 96, "the K block has 96 non-zero entries from 30 tensors");

// The 96 non-zero K entries ordered by input component b, then output a (as kBlockB)
struct KBlockTableB {
    BlockEntryT e[96];
};
constexpr KBlockTableB make_kblock_table_b() {
    KBlockTableB T{};
    int n = 0;
    for (int b = 0; b < 12; ++b)
        for (int a = 0; a < 12; ++a)
            if (kblock::tensor(a, b) >= 0) {
                T.e[n].a = (signed char)a;
                T.e[n].b = (signed char)b;
                T.e[n].t = (signed char)kblock::tensor(a, b);
                T.e[n].s = (signed char)kblock::sign(a, b);
                ++n;
            }
    return T;
}
__device__ constexpr KBlockTableB kKBlockB = make_kblock_table_b();

// ---------------------------------------------------------------------------
// cp.async (shared <- global) helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc));
}
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc));
}
// 8-byte copy that writes zeros when src_bytes == 0 (src must still be a valid address)
__device__ __forceinline__ void cp_async8z(void* smem_dst, const void* gsrc, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// 16-byte zero-filling copy (src_bytes 0 or 16)
__device__ __forceinline__ void cp_async16z(void* smem_dst, const void* gsrc, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(src_bytes));
}
// one element of the input plane: 8-byte (FP32) or 16-byte (FP64) zero-filling copy
template <typename C>
__device__ __forceinline__ void cp_async_elem(C* smem_dst, const C* gsrc, bool in) {
    if constexpr (sizeof(C) == 8)
        cp_async8z(smem_dst, gsrc, in ? 8 : 0);
    else
        cp_async16z(smem_dst, gsrc, in ? 16 : 0);
}

