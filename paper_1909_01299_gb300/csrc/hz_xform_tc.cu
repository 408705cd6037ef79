// Bulk x/y eigen-transforms of the mixed path on the 5th-generation tensor cores.
//
// The transform of steps 1 and 7 of Sec. 2 is, per block, a complex product
// C[rows x n] = A[rows x n] B[n x n] with the block's eigenvector table B
// (forward W^T M or inverse W).  Written over the reals with interleaved
// (re, im) pairs it is one real GEMM of K = N = 2n:
//   A'[row][2a+u] = (Re, Im) of A[row][a],
//   B'[2a][2c] = Re B, B'[2a][2c+1] = Im B, B'[2a+1][2c] = -Im B, B'[2a+1][2c+1] = Re B,
// whose result C' = A' B' is again interleaved complex.  The GEMM runs as
// tcgen05.mma kind::tf32 with FP32 accumulators in tensor memory, in the
// 3xTF32 form A_hi B_hi + A_hi B_lo + A_lo B_hi (x = hi + lo, hi = tf32(x),
// lo = tf32(x - hi)), which keeps the result at FP32 accuracy; FP64 iterative
// refinement of the solve removes the rest.
//
// One CTA (8 warps) computes a 128-row x Nt-column tile (Nt <= 160, a multiple of
// 16) of one block; two CTAs share an SM (108-112 KB of shared memory and 256 TMEM
// columns each).  The contraction runs in chunks of 16 real K (64 bytes per operand
// row): all threads load the data rows (complex128, or complex64 for the mixed path's
// mode-space volumes, which carry FP32 accuracy only) into registers one chunk ahead,
// convert them to TF32 hi/lo and store them in shared memory in the K-major
// 64-byte-swizzled layout (the data never makes a shared-memory round trip before the
// conversion, which spares the shared-memory bandwidth the MMAs need); the tables' hi/lo rows
// arrive in the same layout by one TMA copy per chunk; one thread queues the 6 MMAs of
// the chunk behind those of the previous chunk and commits them to the chunk's
// mbarrier; two operand stages alternate, so the conversion of chunk c+1 overlaps the
// MMAs of chunk c.
// The epilogue reads the accumulator with tcgen05.ld (warp w reads TMEM lanes
// 32(w%4)..+31 = tile rows, column chunks w/4, w/4+2, ...) and stores it as complex128
// (exact) or complex64: transposed outputs straight from registers (a warp's 32 rows are
// consecutive addresses), row-contiguous outputs through an FP32 staging tile in
// shared memory written out row by row; optionally adding to the old values.
// Every mbarrier wait is bounded; on timeout the kernel raises an error flag,
// waits (bounded) for its own MMAs and copies, frees its tensor memory and returns.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda.h>   // CUtensorMap and its enums; the encoder is fetched from the driver at run time

#include "hz_convert.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

constexpr int TC_M = 128;
constexpr int TC_THREADS = 256;          // 8 warps; two CTAs per SM overlap each other's phases
constexpr int TC_CTAS_PER_SM = 2;
constexpr int KCH = 16;                  // real K per chunk (64 bytes of tf32 per operand row)
constexpr int ROWB = 64;                 // bytes per operand row in a chunk (64-byte swizzle)
constexpr int A_BYTES = TC_M * ROWB;     // one A plane (hi or lo) of a chunk
constexpr int TMEM_COLS = 256;           // two CTAs per SM share the 512 columns
constexpr int kTcMaxN = 160;             // widest output tile (real columns)
constexpr long long WAIT_NS = 2000000000LL;   // 2 s bound on any wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  // clock64 counts SM cycles; 2e9 ns at <= 2.1 GHz is < 4.2e9 cycles
  while (!mbar_test(bar, parity)) {
    if (clock64() - t0 > 2 * WAIT_NS) return false;
  }
  return true;
}

// Shared-memory matrix descriptor of a K-major operand with 64-byte rows and the 64-byte
// swizzle (16-byte unit u of row r stored at unit u ^ ((r >> 1) & 3)); 8-row groups are
// 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);          // start address
  d |= (uint64_t)1u << 16;                          // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((512u >> 4) & 0x3FFFu) << 32;     // stride byte offset: 8 rows x 64 B
  d |= (uint64_t)1u << 46;                          // descriptor version
  d |= (uint64_t)4u << 61;                          // 64-byte swizzle
  return d;
}
__device__ __forceinline__ uint32_t swz64(int r, int u) { return (uint32_t)(r * ROWB + ((u ^ ((r >> 1) & 3)) << 4)); }

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Arrive on the barrier (this thread) and add bytes to its expected transaction count.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// 3-D tiled TMA load (tensor map in global memory) completing on an mbarrier.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void* tmap, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory plan of one CTA (offsets from a 1024-byte aligned base):
//   raw[2]   : unused by the chunk loop (the data goes to registers); with the pipeline
//              buffers after it, room for the epilogue's FP32 staging tile
//   aop[2]   : TF32 hi | lo operand planes of a chunk (2 x 8 KB each), 64B-swizzled
//   bop[NB]  : TF32 hi | lo table planes of a chunk (2 x nt x 64 B each), 64B-swizzled; three
//              stages for complex64 data, two for complex128 (whose raw buffers are larger)
//   bars     : MMA-completion mbarriers of the two operand stages, table-arrival mbarriers of
//              the table stages, TMEM address slot
// The chunk pipeline: while chunk c is converted, the MMAs of chunk c-1 run (those of chunk c
// are queued behind them as soon as c is converted), the table rows of chunk c are in flight
// (one TMA copy per chunk: a 16 x nt x 2 box of the tile's 3-D tensor map [plane][row][k]
// with the 64-byte swizzle, which lands in exactly the operand layout above) and so are the
// data rows of chunk c+1 (plain loads into registers: a block may start at any column, so
// its rows have no 16-byte alignment a TMA box would need).
constexpr int RAW_ROWB = KCH * 8;        // FP64 bytes of a data row in a chunk (KCH / 2 complex)
constexpr int RAW_BYTES = TC_M * RAW_ROWB;
__host__ __device__ constexpr int nbstages(bool in32) { return in32 ? 3 : 2; }
__host__ __device__ constexpr int raw_bytes(bool in32) { return in32 ? RAW_BYTES / 2 : RAW_BYTES; }

// TI / TO: double2 (complex128) or float2 (complex64) input / output elements.  NP: TF32
// products per chunk, 3 (3xTF32: A_hi B_hi + A_hi B_lo + A_lo B_hi) or 1 (plain TF32: A_hi B_hi,
// the data's lo plane is neither formed nor read).
template <typename TI, typename TO, int NP>
__global__ void __launch_bounds__(TC_THREADS, TC_CTAS_PER_SM)
xform_tc_kernel(const TI* __restrict__ in, TO* __restrict__ out, const TCBlock* __restrict__ blocks,
                const TCTile* __restrict__ tiles, const unsigned char* __restrict__ tmaps, int ntiles,
                long long nrows, int rows_per_plane, int ncols, int trans, int store,
                const signed char* __restrict__ rowskip, int* __restrict__ err) {
  extern __shared__ uint8_t smem_dyn[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  // column tiles of one row tile are consecutive CTAs (the data rows come from L2 the second time)
  const int tile = (int)(blockIdx.x % ntiles);
  const TCTile t = tiles[tile];
  const void* tmap = tmaps + (size_t)tile * 128;           // this tile's 128-byte tensor map
  const TCBlock b = blocks[t.blk];
  const long long row0 = (long long)(blockIdx.x / ntiles) * TC_M;
  const int nt = t.nt;
  const int B_BYTES = nt * ROWB;                           // one table plane of a chunk
  constexpr bool IN32 = sizeof(TI) == 8, OUT32 = sizeof(TO) == 8;
  constexpr int RAWB = raw_bytes(IN32), NB = nbstages(IN32);
  const uint32_t s_base = smem_u32(smem);
  const uint32_t raw0 = s_base, aop0 = raw0 + 2 * RAWB, bop0 = aop0 + 2 * 2 * A_BYTES;
  const uint32_t BSTAGE = 2 * B_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * RAWB + 4 * A_BYTES + NB * BSTAGE);
  uint64_t* tbars = bars + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 + NB);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = b.size;
  const int nk = b.kpad / KCH;

  // the data values of chunk c that this thread converts: conversion task q (row r = task / 4,
  // 16-byte TF32 unit u = task % 4) needs the complex columns 2u and 2u + 1 of the chunk;
  // loaded straight into registers one chunk ahead (no shared-memory round trip)
  constexpr int NTASK = TC_M * (ROWB / 16) / TC_THREADS;
  TI dreg[NTASK][2];
  auto load_regs = [&](int c) {
#pragma unroll
    for (int q = 0; q < NTASK; ++q) {
      const int task = tid + TC_THREADS * q;
      const int r = task >> 2, u = task & 3;
      const long long grow = row0 + r;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int col = c * (KCH / 2) + 2 * u + h;
        TI v;
        if constexpr (IN32) v = make_float2(0.f, 0.f);
        else v = make_double2(0.0, 0.0);
        if (grow < nrows && col < n) v = __ldg(in + grow * (long long)ncols + b.start + col);
        dreg[q][h] = v;
      }
    }
  };
  // (thread 0) one TMA copy of the table rows (hi and lo planes) of chunk c into bop[c % NB]
  auto load_b = [&](int c) {
    uint64_t* tb = &tbars[c % NB];
    mbar_expect_tx(tb, (uint32_t)(2 * B_BYTES));
    tma_load_3d(bop0 + (c % NB) * BSTAGE, tmap, c * KCH, t.n0, 0, tb);
  };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    for (int q = 0; q < NB; ++q) mbar_init(&tbars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    load_b(0);
  }
  // prologue: data of chunk 0 into registers; table chunk 0 by TMA
  load_regs(0);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_tf32(nt);
  bool ok = true;
  int issued = 0;

  // Iteration kc: (1) wait for the MMAs of kc-2, the last reader of operand stage kc & 1;
  // (2) convert this thread's data values of chunk kc (in registers) into that stage (the
  // MMAs of kc-1 run meanwhile) and start loading those of kc+1 into the same registers;
  // (3) thread 0 waits for the table rows of kc, (4) queues the MMAs of kc behind those of
  // kc-1 and (5) issues the TMA copy of the table rows of kc+1 into stage (kc+1) % NB, last
  // read by the MMAs of kc+1-NB (with two stages: kc-1, which thread 0 waits for first).
  int tab_issued = (tid == 0) ? 1 : 0, tab_done = 0;        // (thread 0) table copies issued / arrived
  for (int kc = 0; kc < nk; ++kc) {
    const int s = kc & 1;
    int w = 1;
    if (kc >= 2) w = mbar_wait(&bars[s], ((kc - 2) >> 1) & 1) ? 1 : 0;
    if (!__syncthreads_and(w)) { ok = false; break; }       // every thread's rows in; stage s free
    {
      const uint32_t a_hi = aop0 + s * 2 * A_BYTES, a_lo = a_hi + A_BYTES;
#pragma unroll
      for (int q = 0; q < NTASK; ++q) {
        const int task = tid + TC_THREADS * q;             // row = task / 4, 16-byte unit = task % 4
        const int r = task >> 2, c = task & 3;
        float f[4];
        if constexpr (IN32) {
          f[0] = dreg[q][0].x;
          f[1] = dreg[q][0].y;
          f[2] = dreg[q][1].x;
          f[3] = dreg[q][1].y;
        } else {
          f[0] = f64_to_f32_trunc(dreg[q][0].x);
          f[1] = f64_to_f32_trunc(dreg[q][0].y);
          f[2] = f64_to_f32_trunc(dreg[q][1].x);
          f[3] = f64_to_f32_trunc(dreg[q][1].y);
        }
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          h[e] = to_tf32(f[e]);
          if (NP == 3) l[e] = to_tf32(f[e] - __uint_as_float(h[e]));
        }
        const uint32_t off = swz64(r, c);
        st_shared_v4(a_hi + off, h[0], h[1], h[2], h[3]);
        if (NP == 3) st_shared_v4(a_lo + off, l[0], l[1], l[2], l[3]);
      }
    }
    if (kc + 1 < nk) load_regs(kc + 1);                    // lands while chunk kc's MMAs run
    int w2 = 1;
    if (tid == 0) {
      if (tab_done < tab_issued && mbar_wait(&tbars[kc % NB], (kc / NB) & 1)) tab_done = kc + 1;
      if (tab_done != kc + 1) w2 = 0;                       // table rows of kc missing
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!__syncthreads_and(w2)) { ok = false; break; }      // operands of kc ready
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = aop0 + s * 2 * A_BYTES, a_lo = a_hi + A_BYTES;
      const uint32_t b_hi = bop0 + (kc % NB) * BSTAGE, b_lo = b_hi + B_BYTES;
#pragma unroll
      for (int ks = 0; ks < KCH / 8; ++ks) {               // 8 tf32 = 32 bytes per MMA
        const uint32_t koff = ks * 32;
        const uint64_t dah = smem_desc_sw64(a_hi + koff), dal = smem_desc_sw64(a_lo + koff);
        const uint64_t dbh = smem_desc_sw64(b_hi + koff), dbl = smem_desc_sw64(b_lo + koff);
        const uint32_t first = (kc == 0 && ks == 0) ? 0u : 1u;
        mma_tf32(tmem, dah, dbh, idesc, first);
        if (NP == 3) {
          mma_tf32(tmem, dah, dbl, idesc, 1u);
          mma_tf32(tmem, dal, dbh, idesc, 1u);
        }
      }
      mma_commit(&bars[s]);
      if (kc + 1 < nk) {
        // the stage of table chunk kc+1 was last read by the MMAs of kc+1-NB: with three
        // stages those of kc-2, waited for in (1); with two those of kc-1
        bool free_stage = true;
        if (NB == 2 && kc >= 1) free_stage = mbar_wait(&bars[(kc - 1) & 1], ((kc - 1) >> 1) & 1);
        if (free_stage) { load_b(kc + 1); tab_issued = kc + 2; }
      }
    }
    issued = kc + 1;
  }
  // (thread 0) a table copy that has not arrived (no later one was issued): wait for it once
  // more, bounded, before the shared memory is given up
  if (tid == 0 && tab_done < tab_issued) {
    const int c = tab_issued - 1;
    mbar_wait(&tbars[c % NB], (c / NB) & 1);
  }
  if (issued > 0) {
    const int last = issued - 1;
    if (!mbar_wait(&bars[last & 1], (last >> 1) & 1)) ok = false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int all_ok = __syncthreads_and(ok ? 1 : 0);
  if (all_ok) {
    const int lw = warp & 3, cgrp = warp >> 2;             // TMEM lane quarter, column group
    constexpr int NGRP = TC_THREADS / 128;
    const int r = lw * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(lw * 32) << 16);
    if (trans) {
      // out[plane][col][row]: the 32 rows of a warp are consecutive addresses of one column
      const long long grow = row0 + r;
      long long plane = 0;
      int rip = 0;
      bool row_ok = grow < nrows;
      if (row_ok) {
        plane = grow / rows_per_plane;
        rip = (int)(grow - plane * rows_per_plane);
        if (rowskip && rowskip[rip]) row_ok = false;
      }
      for (int c16 = 16 * cgrp; c16 < nt; c16 += 16 * NGRP) {
        float v[16];
        tmem_ld16(tl + c16, v);
        if (!row_ok) continue;
        TO* p[8];
        TO val[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int ccol = (t.n0 + c16) / 2 + e;             // complex column within the block
          p[e] = ccol < n ? out + plane * (long long)ncols * rows_per_plane +
                                (long long)(b.start + ccol) * rows_per_plane + rip
                          : nullptr;
          if constexpr (OUT32) val[e] = make_float2(v[2 * e], v[2 * e + 1]);
          else val[e] = make_double2(f32_to_f64(v[2 * e]), f32_to_f64(v[2 * e + 1]));
        }
        if constexpr (!OUT32) {
          if (store == XS_ACCUM) {                         // all old values in flight at once
            double2 o[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) o[e] = p[e] ? *p[e] : make_double2(0.0, 0.0);
#pragma unroll
            for (int e = 0; e < 8; ++e) { val[e].x += o[e].x; val[e].y += o[e].y; }
          }
        }
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (p[e]) *p[e] = val[e];
      }
    } else {
      // Rows are contiguous in memory: stage the FP32 accumulator tile in the (now idle)
      // pipeline buffers -- 128 rows x nt floats, row stride padded by 16 bytes so that the
      // row-per-lane writes are conflict-free; nt * 512 + 2048 bytes fit in the buffers
      // (65536 + 256 * nt bytes for complex128 input, 49152 + 384 * nt for complex64) for
      // every nt <= 248 -- then each warp writes
      // whole rows, consecutive lanes on consecutive complex columns, converting to FP64.
      const int sstride = nt * 4 + 16;
      for (int c16 = 16 * cgrp; c16 < nt; c16 += 16 * NGRP) {
        float v[16];
        tmem_ld16(tl + c16, v);
        const uint32_t dst = s_base + (uint32_t)(r * sstride + c16 * 4);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          st_shared_v4(dst + 16 * q, __float_as_uint(v[4 * q]), __float_as_uint(v[4 * q + 1]),
                       __float_as_uint(v[4 * q + 2]), __float_as_uint(v[4 * q + 3]));
      }
      __syncthreads();
      const int cbase = t.n0 / 2;                           // first complex column of the tile in the block
      const int ccount = min(nt / 2, n - cbase);
      // warp w writes rows w, w + 8, ..., RB rows at a time; with accumulation the old values of
      // the RB rows are all loaded before the first store
      constexpr int NW = TC_THREADS / 32;
      constexpr int CPL = kTcMaxN / 2 / 32 + 1;             // complex columns per lane (<= 3)
      constexpr int RB = 2;
      for (int m0 = 0; m0 < TC_M / NW; m0 += RB) {
        TO* dg[RB];
        const float2* src[RB];
#pragma unroll
        for (int i = 0; i < RB; ++i) {
          const int rr = warp + NW * (m0 + i);
          const long long g = row0 + rr;
          bool rok = g < nrows;
          if (rok && rowskip) {
            const long long pl = g / rows_per_plane;
            rok = rowskip[g - pl * rows_per_plane] == 0;
          }
          dg[i] = rok ? out + g * (long long)ncols + b.start + cbase : nullptr;
          src[i] = reinterpret_cast<const float2*>(smem + (size_t)rr * sstride);
        }
        if constexpr (OUT32) {
#pragma unroll
          for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
              const int c = lane + 32 * q;
              if (dg[i] && c < ccount) dg[i][c] = src[i][c];
            }
        } else if (store == XS_ACCUM) {
          double2 o[RB][CPL];
#pragma unroll
          for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
              const int c = lane + 32 * q;
              if (dg[i] && c < ccount) o[i][q] = dg[i][c];
            }
#pragma unroll
          for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
              const int c = lane + 32 * q;
              if (dg[i] && c < ccount) {
                const float2 f = src[i][c];
                dg[i][c] = make_double2(f32_to_f64(f.x) + o[i][q].x, f32_to_f64(f.y) + o[i][q].y);
              }
            }
        } else {
#pragma unroll
          for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
              const int c = lane + 32 * q;
              if (dg[i] && c < ccount) {
                const float2 f = src[i][c];
                dg[i][c] = make_double2(f32_to_f64(f.x), f32_to_f64(f.y));
              }
            }
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, (int)HZ_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// ---------------------------------------------------------------------------
// Real-table kernel.  When a block's table B is real, C = A B for complex data A is two real
// products, Re C = Re A B and Im C = Im A B.  The MMA rows are the data rows' parts
// (MMA row m = 2 r + u: data row r, u = 0 real / 1 imaginary part), K = N = n (half of the
// interleaved form's 2n each way: a quarter of its MMA work per MMA row, half per data
// row).  One CTA (4 warps) takes 64 data rows x nt <= 128 columns: 128 TMEM
// columns and about 53 KB of shared memory, so four CTAs share an SM.  The chunk loop is the
// interleaved kernel's (16 K per chunk, data in registers one chunk ahead, two operand stages,
// one TMA copy of the table rows per chunk); in the epilogue each lane pair (2r, 2r+1) trades
// half of its columns so that every lane writes whole complex values.
// ---------------------------------------------------------------------------
constexpr int TCR_THREADS = 128;
constexpr int TCR_ROWS = TC_M / 2;                  // data rows per CTA
constexpr int TCR_TMEM = 128;                       // TMEM columns (nt <= 128)
// widest real tile: the epilogue's staging tile (64 rows x (8 nt + 16) bytes) then fits in the
// pipeline buffers below the mbarriers (32768 + 256 nt bytes) for every nt <= 112
constexpr int kTcrMaxN = 112;
constexpr int TCR_CTAS_PER_SM = 4;

template <typename TI, typename TO, int NP>
__global__ void __launch_bounds__(TCR_THREADS, TCR_CTAS_PER_SM)
xform_tcr_kernel(const TI* __restrict__ in, TO* __restrict__ out, const TCBlock* __restrict__ blocks,
                 const TCTile* __restrict__ tiles, const unsigned char* __restrict__ tmaps, int ntiles,
                 long long nrows, int rows_per_plane, int ncols, int trans, int store,
                 const signed char* __restrict__ rowskip, int* __restrict__ err) {
  extern __shared__ uint8_t smem_dyn[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  const int tile = (int)(blockIdx.x % ntiles);
  const TCTile t = tiles[tile];
  const void* tmap = tmaps + (size_t)tile * 128;
  const TCBlock b = blocks[t.blk];
  const long long row0 = (long long)(blockIdx.x / ntiles) * TCR_ROWS;
  const int nt = t.nt;
  const int B_BYTES = nt * ROWB;
  constexpr bool IN32 = sizeof(TI) == 8, OUT32 = sizeof(TO) == 8;
  constexpr int NB = 2;
  const uint32_t s_base = smem_u32(smem);
  const uint32_t aop0 = s_base, bop0 = aop0 + 2 * 2 * A_BYTES;
  const uint32_t BSTAGE = 2 * B_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 4 * A_BYTES + NB * BSTAGE);
  uint64_t* tbars = bars + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 + NB);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = b.size;
  const int nk = b.kpad_r / KCH;

  // conversion task q: data row r = task / 4, complex columns 4 u .. 4 u + 3 of the chunk (u = task
  // % 4) -> one 16-byte TF32 unit of MMA row 2 r (real parts) and of row 2 r + 1 (imaginary)
  constexpr int NTASK = TCR_ROWS * (KCH / 4) / TCR_THREADS;
  TI dreg[NTASK][4];
  auto load_regs = [&](int c) {
#pragma unroll
    for (int q = 0; q < NTASK; ++q) {
      const int task = tid + TCR_THREADS * q;
      const int r = task >> 2, u = task & 3;
      const long long grow = row0 + r;
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int col = c * KCH + 4 * u + h;
        TI v;
        if constexpr (IN32) v = make_float2(0.f, 0.f);
        else v = make_double2(0.0, 0.0);
        if (grow < nrows && col < n) v = __ldg(in + grow * (long long)ncols + b.start + col);
        dreg[q][h] = v;
      }
    }
  };
  auto load_b = [&](int c) {
    uint64_t* tb = &tbars[c % NB];
    mbar_expect_tx(tb, (uint32_t)(2 * B_BYTES));
    tma_load_3d(bop0 + (c % NB) * BSTAGE, tmap, c * KCH, t.n0, 0, tb);
  };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TCR_TMEM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    for (int q = 0; q < NB; ++q) mbar_init(&tbars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    load_b(0);
  }
  load_regs(0);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_tf32(nt);
  bool ok = true;
  int issued = 0;
  int tab_issued = (tid == 0) ? 1 : 0, tab_done = 0;
  // iteration kc as in the interleaved kernel: (1) MMAs of kc-2 done (stage kc & 1 free);
  // (2) convert chunk kc from registers, start loading kc+1; (3) table rows of kc arrived;
  // (4) queue the MMAs of kc; (5) table rows of kc+1 into the stage the MMAs of kc-1 read
  for (int kc = 0; kc < nk; ++kc) {
    const int s = kc & 1;
    int w = 1;
    if (kc >= 2) w = mbar_wait(&bars[s], ((kc - 2) >> 1) & 1) ? 1 : 0;
    if (!__syncthreads_and(w)) { ok = false; break; }
    {
      const uint32_t a_hi = aop0 + s * 2 * A_BYTES, a_lo = a_hi + A_BYTES;
#pragma unroll
      for (int q = 0; q < NTASK; ++q) {
        const int task = tid + TCR_THREADS * q;
        const int r = task >> 2, u = task & 3;
        float fr[4], fi[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          if constexpr (IN32) {
            fr[h] = dreg[q][h].x;
            fi[h] = dreg[q][h].y;
          } else {
            fr[h] = f64_to_f32_trunc(dreg[q][h].x);
            fi[h] = f64_to_f32_trunc(dreg[q][h].y);
          }
        }
        uint32_t hr[4], lr[4], hi[4], li[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          hr[h] = to_tf32(fr[h]);
          hi[h] = to_tf32(fi[h]);
          if (NP == 3) {
            lr[h] = to_tf32(fr[h] - __uint_as_float(hr[h]));
            li[h] = to_tf32(fi[h] - __uint_as_float(hi[h]));
          }
        }
        const uint32_t offr = swz64(2 * r, u), offi = swz64(2 * r + 1, u);
        st_shared_v4(a_hi + offr, hr[0], hr[1], hr[2], hr[3]);
        st_shared_v4(a_hi + offi, hi[0], hi[1], hi[2], hi[3]);
        if (NP == 3) {
          st_shared_v4(a_lo + offr, lr[0], lr[1], lr[2], lr[3]);
          st_shared_v4(a_lo + offi, li[0], li[1], li[2], li[3]);
        }
      }
    }
    if (kc + 1 < nk) load_regs(kc + 1);
    int w2 = 1;
    if (tid == 0) {
      if (tab_done < tab_issued && mbar_wait(&tbars[kc % NB], (kc / NB) & 1)) tab_done = kc + 1;
      if (tab_done != kc + 1) w2 = 0;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!__syncthreads_and(w2)) { ok = false; break; }
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = aop0 + s * 2 * A_BYTES, a_lo = a_hi + A_BYTES;
      const uint32_t b_hi = bop0 + (kc % NB) * BSTAGE, b_lo = b_hi + B_BYTES;
#pragma unroll
      for (int ks = 0; ks < KCH / 8; ++ks) {
        const uint32_t koff = ks * 32;
        const uint64_t dah = smem_desc_sw64(a_hi + koff), dal = smem_desc_sw64(a_lo + koff);
        const uint64_t dbh = smem_desc_sw64(b_hi + koff), dbl = smem_desc_sw64(b_lo + koff);
        const uint32_t first = (kc == 0 && ks == 0) ? 0u : 1u;
        mma_tf32(tmem, dah, dbh, idesc, first);
        if (NP == 3) {
          mma_tf32(tmem, dah, dbl, idesc, 1u);
          mma_tf32(tmem, dal, dbh, idesc, 1u);
        }
      }
      mma_commit(&bars[s]);
      if (kc + 1 < nk) {
        bool free_stage = true;
        if (kc >= 1) free_stage = mbar_wait(&bars[(kc - 1) & 1], ((kc - 1) >> 1) & 1);
        if (free_stage) { load_b(kc + 1); tab_issued = kc + 2; }
      }
    }
    issued = kc + 1;
  }
  if (tid == 0 && tab_done < tab_issued) {
    const int c = tab_issued - 1;
    mbar_wait(&tbars[c % NB], (c / NB) & 1);
  }
  if (issued > 0) {
    const int last = issued - 1;
    if (!mbar_wait(&bars[last & 1], (last >> 1) & 1)) ok = false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int all_ok = __syncthreads_and(ok ? 1 : 0);
  if (all_ok) {
    // TMEM lane m = 32 warp + lane holds MMA row m: data row r = m / 2, part = m % 2
    const int m = warp * 32 + lane;
    const int r = m >> 1;
    const bool odd = (lane & 1) != 0;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    const long long grow = row0 + r;
    bool row_ok = grow < nrows;
    long long plane = 0;
    int rip = 0;
    if (row_ok) {
      plane = grow / rows_per_plane;
      rip = (int)(grow - plane * rows_per_plane);
      if (rowskip && rowskip[rip]) row_ok = false;
    }
    if (!trans) {
      // rows are contiguous in memory: stage the tile as complex64 (row stride 8 nt + 16 bytes)
      // in the idle pipeline buffers, then each warp writes whole rows, consecutive lanes on
      // consecutive columns
      const int sstride = nt * 8 + 16;
      for (int c16 = 0; c16 < nt; c16 += 16) {
        float v[16];
        tmem_ld16(tl + c16, v);
        float* dst = reinterpret_cast<float*>(smem + (size_t)r * sstride) + 2 * c16 + (odd ? 1 : 0);
#pragma unroll
        for (int e = 0; e < 16; ++e) dst[2 * e] = v[e];
      }
      __syncthreads();
      const int ccount = min(nt, n - t.n0);
      // warp w writes rows w, w + 4, ..., RB rows at a time: with accumulation the old values of
      // the RB rows are all loaded before the first store (a store may alias a later load, so
      // the compiler keeps them in program order: row by row, each old value would cost a
      // full memory latency)
      constexpr int NW = TCR_THREADS / 32;
      constexpr int CPL = kTcrMaxN / 32 + 1;              // complex columns per lane (<= 4)
      constexpr int RB = 4;
      for (int m0 = 0; m0 < TCR_ROWS / NW; m0 += RB) {
        TO* dg[RB];
        const float2* srow[RB];
#pragma unroll
        for (int i = 0; i < RB; ++i) {
          const int rr = warp + NW * (m0 + i);
          const long long g = row0 + rr;
          bool rok = g < nrows;
          if (rok && rowskip) {
            const long long pl = g / rows_per_plane;
            rok = rowskip[g - pl * rows_per_plane] == 0;
          }
          dg[i] = rok ? out + g * (long long)ncols + b.start + t.n0 : nullptr;
          srow[i] = reinterpret_cast<const float2*>(smem + (size_t)rr * sstride);
        }
        if constexpr (OUT32) {
#pragma unroll
          for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
              const int c = lane + 32 * q;
              if (dg[i] && c < ccount) dg[i][c] = srow[i][c];
            }
        } else if (store == XS_ACCUM) {
          double2 o[RB][CPL];
#pragma unroll
          for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
              const int c = lane + 32 * q;
              if (dg[i] && c < ccount) o[i][q] = dg[i][c];
            }
#pragma unroll
          for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
              const int c = lane + 32 * q;
              if (dg[i] && c < ccount) {
                const float2 f = srow[i][c];
                dg[i][c] = make_double2(f32_to_f64(f.x) + o[i][q].x, f32_to_f64(f.y) + o[i][q].y);
              }
            }
        } else {
          // no FP64 arithmetic here: the FP64 pipe is 64x slower than FP32 (an add of zero would
          // cost as much as the accumulation)
#pragma unroll
          for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
              const int c = lane + 32 * q;
              if (dg[i] && c < ccount) {
                const float2 f = srow[i][c];
                dg[i][c] = make_double2(f32_to_f64(f.x), f32_to_f64(f.y));
              }
            }
        }
      }
    }
    for (int c16 = 0; trans && c16 < nt; c16 += 16) {
      float v[16];
      tmem_ld16(tl + c16, v);
      // the even lane (real parts) keeps columns c16..c16+7, the odd lane (imaginary parts) the
      // next eight: each sends the partner's half
      float part[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float send = odd ? v[e] : v[8 + e];
        part[e] = __shfl_xor_sync(0xffffffffu, send, 1);
      }
      if (!row_ok) continue;
      TO* p[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int ccol = t.n0 + c16 + (odd ? 8 : 0) + e;      // complex column within the block
        p[e] = ccol < n ? out + plane * (long long)ncols * rows_per_plane + (long long)(b.start + ccol) * rows_per_plane + rip
                        : nullptr;
      }
      if constexpr (OUT32) {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (p[e]) *p[e] = odd ? make_float2(part[e], v[8 + e]) : make_float2(v[e], part[e]);
      } else if (store == XS_ACCUM) {
        double2 o[8];                                         // all old values in flight at once
#pragma unroll
        for (int e = 0; e < 8; ++e) o[e] = p[e] ? *p[e] : make_double2(0.0, 0.0);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float re = odd ? part[e] : v[e];
          const float im = odd ? v[8 + e] : part[e];
          if (p[e]) *p[e] = make_double2(f32_to_f64(re) + o[e].x, f32_to_f64(im) + o[e].y);
        }
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float re = odd ? part[e] : v[e];
          const float im = odd ? v[8 + e] : part[e];
          if (p[e]) *p[e] = make_double2(f32_to_f64(re), f32_to_f64(im));
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, (int)HZ_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCR_TMEM));
}

size_t xform_tcr_smem(int nt_max) {
  // at least 46 KB, so that no more than four CTAs (TCR_TMEM columns each) share an SM
  const size_t need = 1024 + 4 * (size_t)A_BYTES + 2 * 2 * (size_t)nt_max * ROWB + 64;
  return std::max(need, (size_t)46 * 1024);
}

float tf32_round_host(double x) {
  // round an FP32 value to TF32 (10 explicit mantissa bits), nearest, ties away from zero
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
  memcpy(&f, &u, 4);
  return f;
}

}  // namespace

void tc_pack_block(const cd* B, int n, int start, std::vector<float>& tab, TCBlock& blk,
                   std::vector<TCTile>& tiles, int blk_index, std::vector<TCTile>* real_tiles) {
  blk.start = start;
  blk.size = n;
  blk.npad_r = blk.kpad_r = 0;
  blk.toff_r = 0;
  blk.npad = ((2 * n + 15) / 16) * 16;
  blk.kpad = ((2 * n + KCH - 1) / KCH) * KCH;
  blk.toff = (long long)tab.size();
  const size_t plane = (size_t)blk.npad * blk.kpad;
  tab.resize(tab.size() + 2 * plane, 0.0f);
  float* hi = tab.data() + blk.toff;
  float* lo = hi + plane;
  for (int a = 0; a < n; ++a)
    for (int c = 0; c < n; ++c) {
      const cd v = B[(size_t)a * n + c];
      // B'[2a+u][2c+v]: (0,0) Re, (0,1) Im, (1,0) -Im, (1,1) Re; stored K-major T[2c+v][2a+u]
      const double e[2][2] = {{v.real(), v.imag()}, {-v.imag(), v.real()}};
      for (int u = 0; u < 2; ++u)
        for (int w = 0; w < 2; ++w) {
          const size_t o = (size_t)(2 * c + w) * blk.kpad + (2 * a + u);
          const float h = tf32_round_host(e[u][w]);
          hi[o] = h;
          lo[o] = tf32_round_host(e[u][w] - (double)h);
        }
    }
  const int ntl = (blk.npad + kTcMaxN - 1) / kTcMaxN;     // tiles of at most kTcMaxN columns
  const int units = blk.npad / 16;
  int n0 = 0;
  for (int q = 0; q < ntl; ++q) {
    const int w = 16 * ((units * (q + 1)) / ntl - (units * q) / ntl);
    tiles.push_back(TCTile{blk_index, n0, w, 0});
    n0 += w;
  }
  if (!real_tiles) return;
  // the real form: T[c][a] = B[a][c], K-major, hi then lo; tiles of at most kTcrMaxN columns
  blk.npad_r = ((n + 15) / 16) * 16;
  blk.kpad_r = ((n + KCH - 1) / KCH) * KCH;
  blk.toff_r = (long long)tab.size();
  const size_t rplane = (size_t)blk.npad_r * blk.kpad_r;
  tab.resize(tab.size() + 2 * rplane, 0.0f);
  float* rhi = tab.data() + blk.toff_r;
  float* rlo = rhi + rplane;
  for (int a = 0; a < n; ++a)
    for (int c = 0; c < n; ++c) {
      const double v = B[(size_t)a * n + c].real();
      const size_t o = (size_t)c * blk.kpad_r + a;
      const float h = tf32_round_host(v);
      rhi[o] = h;
      rlo[o] = tf32_round_host(v - (double)h);
    }
  const int rtl = (blk.npad_r + kTcrMaxN - 1) / kTcrMaxN;
  const int runits = blk.npad_r / 16;
  int c0 = 0;
  for (int q = 0; q < rtl; ++q) {
    const int w = 16 * ((runits * (q + 1)) / rtl - (runits * q) / rtl);
    real_tiles->push_back(TCTile{blk_index, c0, w, 0});
    c0 += w;
  }
}

bool tc_encode_tmaps(const float* d_tab, const std::vector<TCBlock>& blocks, const std::vector<TCTile>& tiles,
                     std::vector<unsigned char>& bytes, bool real) {
  using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeTiled encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<EncodeTiled>(fn);
  }
  std::vector<CUtensorMap> maps(tiles.size());
  for (size_t i = 0; i < tiles.size(); ++i) {
    const TCBlock& b = blocks[tiles[i].blk];
    // [plane][row][k] view of the block's hi | lo tables; box = one chunk of K x the tile's rows
    // x both planes, 64-byte swizzle (the K-major operand layout of the MMA descriptors)
    const int kp = real ? b.kpad_r : b.kpad, np = real ? b.npad_r : b.npad;
    if (np == 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)kp, (cuuint64_t)np, 2};
    const cuuint64_t strides[2] = {(cuuint64_t)kp * 4, (cuuint64_t)np * kp * 4};
    const cuuint32_t box[3] = {(cuuint32_t)KCH, (cuuint32_t)tiles[i].nt, 2};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (encode(&maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(d_tab + (real ? b.toff_r : b.toff)),
               dims, strides,
               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  static_assert(sizeof(CUtensorMap) == 128, "tensor maps are 128 bytes");
  bytes.resize(maps.size() * sizeof(CUtensorMap));
  if (!maps.empty()) std::memcpy(bytes.data(), maps.data(), bytes.size());
  return true;
}

size_t xform_tc_smem(int nt_max, bool in32) {
  // at least 80 KB, so that no more than TC_CTAS_PER_SM CTAs (each holding TMEM_COLS) share an SM
  const size_t need = 1024 + 2 * (size_t)raw_bytes(in32) + 4 * A_BYTES +
                      (size_t)nbstages(in32) * 2 * nt_max * ROWB + 64;
  return std::max(need, (size_t)80 * 1024);
}

uint32_t xform_tc_idesc(int nt) { return idesc_tf32(nt); }

template <typename TI, typename TO>
void set_smem_attr() {
  cudaFuncSetAttribute(xform_tc_kernel<TI, TO, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)xform_tc_smem(kTcMaxN, sizeof(TI) == 8));
  cudaFuncSetAttribute(xform_tc_kernel<TI, TO, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)xform_tc_smem(kTcMaxN, sizeof(TI) == 8));
  cudaFuncSetAttribute(xform_tcr_kernel<TI, TO, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)xform_tcr_smem(kTcrMaxN));
  cudaFuncSetAttribute(xform_tcr_kernel<TI, TO, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)xform_tcr_smem(kTcrMaxN));
}

void xform_tc_prepare() {
  int dev = 0;
  cudaGetDevice(&dev);
  static bool attr_set[64] = {};
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    // the largest tile any plan uses, so every launch fits
    set_smem_attr<double2, double2>();
    set_smem_attr<double2, float2>();
    set_smem_attr<float2, float2>();
    set_smem_attr<float2, double2>();
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
}

bool xform_tc(const TCSet& ts, const void* in, int in32, void* out, int out32, int rows_per_plane,
              long long nplanes, int trans, int store, const signed char* rowskip, int* err,
              cudaStream_t st, int products, bool skip_fast, bool real_tables) {
  if (out32 && store != XS_STORE) return false;          // accumulation needs a complex128 output
  const int v = (skip_fast ? 1 : 0) + (real_tables ? 2 : 0);
  const TCList& cl = ts.cl[v];
  const TCList& rl = ts.rl[v];
  const long long nrows = nplanes * (long long)rows_per_plane;
  if (nrows <= 0) return true;
  if ((cl.ntiles && !cl.d_tmaps) || (rl.ntiles && !rl.d_tmaps)) return false;
  xform_tc_prepare();
#define HZ_TC_LAUNCH(K, CTAS, THREADS, SMEM, L, TI, TO, NP)                                            \
  K<TI, TO, NP><<<(unsigned)(CTAS), THREADS, SMEM, st>>>(                                              \
      static_cast<const TI*>(in), static_cast<TO*>(out), ts.d_blocks, L.d_tiles, L.d_tmaps, L.ntiles, nrows, \
      rows_per_plane, ts.ncols, trans, store, rowskip, err)
#define HZ_TC_TYPES(K, CTAS, THREADS, SMEM, L)                                                         \
  do {                                                                                                 \
    if (products == 1) {                                                                               \
      if (in32 && out32) HZ_TC_LAUNCH(K, CTAS, THREADS, SMEM, L, float2, float2, 1);                  \
      else if (in32) HZ_TC_LAUNCH(K, CTAS, THREADS, SMEM, L, float2, double2, 1);                     \
      else if (out32) HZ_TC_LAUNCH(K, CTAS, THREADS, SMEM, L, double2, float2, 1);                    \
      else HZ_TC_LAUNCH(K, CTAS, THREADS, SMEM, L, double2, double2, 1);                              \
    } else {                                                                                           \
      if (in32 && out32) HZ_TC_LAUNCH(K, CTAS, THREADS, SMEM, L, float2, float2, 3);                  \
      else if (in32) HZ_TC_LAUNCH(K, CTAS, THREADS, SMEM, L, float2, double2, 3);                     \
      else if (out32) HZ_TC_LAUNCH(K, CTAS, THREADS, SMEM, L, double2, float2, 3);                    \
      else HZ_TC_LAUNCH(K, CTAS, THREADS, SMEM, L, double2, double2, 3);                              \
    }                                                                                                  \
    count_launch();                                                                                    \
  } while (0)
  if (cl.ntiles) {
    const long long ctas = ((nrows + TC_M - 1) / TC_M) * cl.ntiles;
    HZ_TC_TYPES(xform_tc_kernel, ctas, TC_THREADS, xform_tc_smem(cl.nt_max, in32 != 0), cl);
  }
  if (rl.ntiles) {
    const long long ctas = ((nrows + TCR_ROWS - 1) / TCR_ROWS) * rl.ntiles;
    HZ_TC_TYPES(xform_tcr_kernel, ctas, TCR_THREADS, xform_tcr_smem(rl.nt_max), rl);
  }
#undef HZ_TC_TYPES
#undef HZ_TC_LAUNCH
  return true;
}

}  // namespace hz
