// bf16xN GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// C = alpha * Z + beta * C with Z the sum of the mode's bfloat16 piece
// products (Sec. II-D, II-G of the paper):
//   x1: a0 b0;  x3: + a0 b1 + a1 b0;  x6: + a0 b2 + a1 b1 + a2 b0;
//   x8: + a1 b2 + a2 b1 (the Z3 sum of Sec. II-D);  x9: all;
//   x5: A split in two pieces, B in three (Sec. II-G's asymmetric case):
//       a0 b0, a0 b1, a1 b0, a0 b2, a1 b1.
// Each product of two bfloat16 values is exact in FP32 (Sec. I) and the
// tensor core accumulates in FP32, the precision the paper's FMA model uses.
//
// Accumulation layout.  Two FP32 accumulators per output tile live in tensor
// memory: D_main receives the hi*hi product (the 2^0 bin) and D_corr every
// correction product.  Within each K-slice the corrections are issued from
// the smallest bin to the largest (2^-32, 2^-24, 2^-16, 2^-8), as Sec. II-G
// prescribes, and the epilogue forms Z = D_main + D_corr in FP32, the
// "Z0 + (Z1 + Z2)" combination of Sec. II-D.  Keeping the small products out
// of the large accumulator means their rounding errors are relative to the
// correction's magnitude (~2^-8 |Z|), not to |Z|.
//
// Kernel structure (one CTA per SM, persistent over output tiles):
//   warp 0    TMA producer: per K-slice one 3-D bulk-tensor load brings all
//             pieces of the A tile and one all pieces of the B tile (the piece
//             index is the third tensor dimension) into a 64/128-byte
//             swizzled, K-major shared-memory stage; completion on `full`.
//   warp 1    MMA issuer (one thread): tcgen05.mma kind::f16, M=128, N=BN,
//             K=16, A and B from shared-memory descriptors, D in tensor memory;
//             tcgen05.commit releases the stage (`empty`) and, after the last
//             slice, hands the accumulator to the epilogue (`acc_full`).
//   warps 2-5 epilogue: tcgen05.ld of both accumulators (each warp owns the
//             32 tensor-memory lanes = tile rows its warp id selects), sum,
//             alpha/beta, store; releases the accumulator (`acc_empty`) as
//             soon as it has been read so the next tile's MMAs overlap the
//             stores.
// FP64-collection variant (D64 = true, the "d" of Sec. IV-A): every product
// gets its own FP32 accumulator in tensor memory and the epilogue adds the
// partial products in FP64, in Sec. II-D's order (Z1 = Z01 + Z10,
// Z2 = Z02 + (Z11 + Z20), Z3 = Z12 + Z21, Z4 = Z22, Z = Z0 + (Z1 + (Z2 + (Z3 +
// Z4)))), and stores C in FP64 without a final rounding to FP32.
// Fused variant (FUSED = true): warp 0 loads FP32 tiles of A (128 x 16) and
// B (16 x BN) by TMA into a ring of FP32 stages; sixteen converter warps split
// each element in registers into its bfloat16 pieces (the same per-element
// split as the separate pass, Sec. II-A) and store them, already in the
// swizzled K-major layout the MMA descriptors expect, into the piece stages;
// the MMA and epilogue roles are unchanged.  No piece buffer in global memory
// is needed, and the results equal those of the separate split + GEMM bit for
// bit (same pieces, same MMA sequence).
// Every mbarrier wait is bounded; on expiry the kernel records an error code
// in the device error word and all roles leave their loops, drain the
// in-flight copies/MMAs (again with a bound) and free tensor memory.
#include <cudaTypedefs.h>

#include "bfx_internal.cuh"

namespace bfx {
namespace {

constexpr int BM = 128;     // UMMA M (one CTA, cta_group::1)
// Long-K accuracy: beyond kChunkMinK the hi*hi product is accumulated in
// chunks of kChunkK (a fresh tensor-memory accumulation each chunk) and the
// chunk sums are added in FP32 with round to nearest by the epilogue.  The
// tensor core adds each 16-deep block into its FP32 accumulator without
// round-to-nearest, so over a long K the hi*hi accumulator's error grows
// with the number of blocks; chunking bounds that growth to kChunkK / 16
// blocks and leaves the rest to round-to-nearest additions.
constexpr int kChunkK = 256;
constexpr int kChunkMinK = 512;
constexpr int GROUP_M = 16; // tile raster: groups of 16 row-blocks for L2 reuse

struct Prod {
  int a, b, acc;  // piece of A, piece of B, accumulator (0 = main, 1 = correction)
};

// pieces of A and of B the mode reads
__host__ __device__ constexpr int mode_npa(int mode) {
  return mode == 1 ? 1 : ((mode == 3 || mode == 5) ? 2 : 3);
}
__host__ __device__ constexpr int mode_npb(int mode) { return mode == 1 ? 1 : (mode == 3 ? 2 : 3); }

// Issue order of the products: corrections smallest bin first, hi*hi last.
__host__ __device__ constexpr Prod prod_of(int mode, int i) {
  if (mode == 1) return Prod{0, 0, 0};
  if (mode == 3) {
    const Prod p[3] = {{1, 0, 1}, {0, 1, 1}, {0, 0, 0}};
    return p[i];
  }
  if (mode == 5) {
    const Prod p[5] = {{0, 2, 1}, {1, 1, 1}, {1, 0, 1}, {0, 1, 1}, {0, 0, 0}};
    return p[i];
  }
  if (mode == 6) {
    const Prod p[6] = {{2, 0, 1}, {1, 1, 1}, {0, 2, 1}, {1, 0, 1}, {0, 1, 1}, {0, 0, 0}};
    return p[i];
  }
  if (mode == 8) {
    const Prod p[8] = {{2, 1, 1}, {1, 2, 1}, {2, 0, 1}, {1, 1, 1},
                       {0, 2, 1}, {1, 0, 1}, {0, 1, 1}, {0, 0, 0}};
    return p[i];
  }
  const Prod p[9] = {{2, 2, 1}, {2, 1, 1}, {1, 2, 1}, {2, 0, 1}, {1, 1, 1},
                     {0, 2, 1}, {1, 0, 1}, {0, 1, 1}, {0, 0, 0}};
  return p[i];
}
// Index of product (a, b) in the mode's issue order (-1 if unused); with
// D64 it is also the product's accumulator.
__host__ __device__ constexpr int prod_slot(int mode, int a, int b) {
  for (int i = 0; i < mode; ++i)
    if (prod_of(mode, i).a == a && prod_of(mode, i).b == b) return i;
  return -1;
}
// Is product i the first one written into its accumulator?
__host__ __device__ constexpr bool first_in_acc(int mode, int i) {
  for (int j = 0; j < i; ++j)
    if (prod_of(mode, j).acc == prod_of(mode, i).acc) return false;
  return true;
}

struct TcArgs {
  int M, N, K;
  int tiles_m, tiles_n, num_tiles, k_tiles;
  float alpha, beta;
  float* C;
  double* Cd;  // D64: the FP64 result (alpha, beta unused)
  int64_t ldc;
  int vec_c;  // C rows 16-byte aligned: float4 (double2) loads/stores
  int* err;
  // grouped mode: many independent problems in one launch
  const GroupTile* tiles;   // num_tiles entries
  const GroupProblem* probs;
};

// What one output tile needs, in both modes.
struct TileInfo {
  int mb, nb, k_tiles, c2, M, N;
  float* C;
  int64_t ldc;
  int vec_c;
};

template <bool GROUPED>
__device__ __forceinline__ TileInfo get_tile(int t, const TcArgs& a);

__device__ __forceinline__ void tile_coords(int t, const TcArgs& a, int& mb, int& nb) {
  const int group = GROUP_M * a.tiles_n;
  const int g = t / group;
  const int first_m = g * GROUP_M;
  const int gm = min(a.tiles_m - first_m, GROUP_M);
  const int r = t - g * group;
  mb = first_m + r % gm;
  nb = r / gm;
}

template <>
__device__ __forceinline__ TileInfo get_tile<false>(int t, const TcArgs& a) {
  TileInfo ti;
  tile_coords(t, a, ti.mb, ti.nb);
  ti.k_tiles = a.k_tiles;
  ti.c2 = 0;
  ti.M = a.M;
  ti.N = a.N;
  ti.C = a.C;
  ti.ldc = a.ldc;
  ti.vec_c = a.vec_c;
  return ti;
}

// Grouped mode: tile t of the list belongs to problem tiles[t].prob; the
// pieces of problem p are planes p*np .. p*np+np-1 of the packed buffers.
template <>
__device__ __forceinline__ TileInfo get_tile<true>(int t, const TcArgs& a) {
  const GroupTile g = a.tiles[t];
  const GroupProblem pr = a.probs[g.prob];
  TileInfo ti;
  ti.mb = g.mb;
  ti.nb = g.nb;
  ti.k_tiles = pr.k_tiles;
  ti.c2 = pr.plane0;
  ti.M = pr.M;
  ti.N = pr.N;
  ti.C = pr.C;
  ti.ldc = pr.ldc;
  ti.vec_c = pr.vec_c;
  return ti;
}

__host__ __device__ constexpr uint32_t pow2_cols(uint32_t c) {
  uint32_t p = 32;
  while (p < c) p *= 2;
  return p;
}

template <int MODE, int BN, int BK, int STAGES, bool FUSED = false, bool D64 = false, int CH = 0>
struct TcConfig {
  static constexpr int NPA = mode_npa(MODE);
  static constexpr int NPB = mode_npb(MODE);
  static constexpr int NP = NPA;  // fused: both operands alike
  static constexpr int NPROD = MODE;
  // chunked (CH > 0): D_main (restarted every chunk) and D_corr
  static constexpr int NACC = D64 ? MODE : ((MODE == 1) ? 1 : 2);
  static constexpr int ACC_BUFS = CH > 0 ? 1 : ((NACC * BN * 2 <= 512) ? 2 : 1);
  static constexpr uint32_t TMEM_USED = NACC * BN * ACC_BUFS;
  static constexpr uint32_t TMEM_COLS = pow2_cols(TMEM_USED);
  static constexpr int SW = BK * 2;  // swizzle span = bytes of one K-slice row
  static constexpr uint32_t A_TILE = BM * BK * 2;
  static constexpr uint32_t B_TILE = BN * BK * 2;
  static constexpr uint32_t STAGE_A = NPA * A_TILE;
  static constexpr uint32_t STAGE = NPA * A_TILE + NPB * B_TILE;
  // fused: FP32 stages of 16 K-columns (A 128 x 16 with 64-byte swizzle, B 16 x BN plain)
  static constexpr int KF = 16;
  static constexpr uint32_t A32_TILE = BM * KF * 4;
  static constexpr uint32_t STAGE32 = FUSED ? (BM + BN) * KF * 4 : 1;
  // as many FP32 stages as the rest of shared memory holds (up to 8): they
  // carry the loads in flight that hide the memory latency
  static constexpr int S32_FIT = static_cast<int>((232448u - 1280u - STAGES * STAGE) / STAGE32);
  static constexpr int S32 = FUSED ? (S32_FIT < 8 ? S32_FIT : 8) : 0;
  static constexpr int CONV_WARPS = FUSED ? 16 : 0;
  // chunked: four epilogue warps per tensor-memory lane quarter, each holding
  // the running hi*hi sums of a quarter of the tile's columns
  static constexpr int EPI_WARPS = CH > 0 ? 16 : 4;
  static constexpr int THREADS = 64 + 32 * EPI_WARPS + 32 * CONV_WARPS;
  static constexpr uint32_t BAR_BYTES = 256;
  static constexpr uint32_t SMEM = STAGES * STAGE + S32 * STAGE32 + BAR_BYTES + 1024;  // + alignment
  static_assert(SW == 64 || SW == 128, "BK must be 32 or 64 bfloat16");
  static_assert(A32_TILE % 1024 == 0, "FP32 stage parts keep the 1024-byte alignment");
  static_assert(!FUSED || (BK == 32 && BN == 256), "fused: BK 32 (two FP32 stages a K-slice), BN 256");
  static_assert(!FUSED || (NPA == NPB && !D64), "fused: symmetric modes, FP32 result");
  static_assert(TMEM_USED <= 512, "tensor memory: 512 columns");
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N");
  static_assert(SMEM <= 232448, "shared memory");
  static_assert((2 * STAGES + 2 * S32 + 2 * ACC_BUFS + 1 + 4) * 8 + 4 <= BAR_BYTES, "barrier area");
  static_assert(CH == 0 || (!FUSED && !D64 && MODE != 1), "chunked: split pieces, FP32 result");
};

// Converter warps of the fused kernel: split one FP32 stage (16 K-columns)
// into half of a piece stage (K-chunks 2h, 2h+1 of the 32-wide slice).
// Chunk c of row r of a 64-byte-swizzled K-major tile sits at r*64 + 16*(c ^ ((r>>1)&3)).
//
// Fast path: pairs of values through cvt.rn.bf16x2 (two RNE conversions in one
// instruction), remainders by exact FP32 subtraction: bit for bit the split
// of split_elem for every finite value whose RNE bfloat16 does not overflow.
// A warp in which any hi piece comes out with an all-ones exponent (Inf/NaN
// input, or the overflow case of the split's reading R3) redoes its values
// with split_elem.

__device__ __forceinline__ uint32_t cvt_bf16x2(float lo_elem, float hi_elem) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi_elem), "f"(lo_elem));
  return r;
}

// w[p] = (piece p of e1) << 16 | (piece p of e0); returns nonzero if a hi half
// has an all-ones exponent (then the pair needs split_elem).
template <int NP>
__device__ __forceinline__ uint32_t split_pair(float e0, float e1, uint32_t (&w)[3]) {
  const uint32_t h = cvt_bf16x2(e0, e1);
  w[0] = h;
  if (NP >= 2) {
    const float r0 = __fsub_rn(e0, __uint_as_float(h << 16));
    const float r1 = __fsub_rn(e1, __uint_as_float(h & 0xFFFF0000u));
    const uint32_t m = cvt_bf16x2(r0, r1);
    w[1] = m;
    if (NP >= 3) {
      const float s0 = __fsub_rn(r0, __uint_as_float(m << 16));
      const float s1 = __fsub_rn(r1, __uint_as_float(m & 0xFFFF0000u));
      w[2] = cvt_bf16x2(s0, s1);
    }
  }
  return __vcmpeq2(h & 0x7F807F80u, 0x7F807F80u);
}

// Pieces of 8 consecutive values as one 16-byte word per piece.
template <int NP>
__device__ __forceinline__ void split8(const float (&e)[8], uint4 (&o)[3]) {
  uint32_t w[4][3];
  uint32_t bad = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) bad |= split_pair<NP>(e[2 * j], e[2 * j + 1], w[j]);
  if (__any_sync(0xFFFFFFFFu, bad != 0)) {
    uint16_t q[3][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) split_elem(e[i], q[0][i], q[1][i], q[2][i]);
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        w[j][p] = q[p][2 * j] | (static_cast<uint32_t>(q[p][2 * j + 1]) << 16);
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) o[p] = make_uint4(w[0][p], w[1][p], w[2][p], w[3][p]);
}

// Pieces of 4 consecutive values as one 8-byte word per piece.
template <int NP>
__device__ __forceinline__ void split4(const float4 x, uint2 (&o)[3]) {
  uint32_t w[2][3];
  uint32_t bad = split_pair<NP>(x.x, x.y, w[0]) | split_pair<NP>(x.z, x.w, w[1]);
  if (__any_sync(0xFFFFFFFFu, bad != 0)) {
    const float e[4] = {x.x, x.y, x.z, x.w};
    uint16_t q[3][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) split_elem(e[i], q[0][i], q[1][i], q[2][i]);
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int j = 0; j < 2; ++j)
        w[j][p] = q[p][2 * j] | (static_cast<uint32_t>(q[p][2 * j + 1]) << 16);
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) o[p] = make_uint2(w[0][p], w[1][p]);
}

// 16 converter warps, thread ct (0..511).  A: row ct/4, FP32 chunk ct%4 (4
// K-values) -> half of a 16-byte piece chunk.  B: column ct%256, K-values
// 8*(ct/256) .. +7 of the stage -> one 16-byte piece chunk of row n of B^T
// (a warp reads 32 consecutive columns: no bank conflicts).
template <int NP, int BN>
__device__ __forceinline__ void convert_half(const uint8_t* st32, uint8_t* pst, int h, int ct) {
  constexpr uint32_t A_TILE = BM * 32 * 2, B_TILE = BN * 32 * 2, A32_TILE = BM * 16 * 4;
  {  // A: FP32 rows of 16 values (64 bytes, 64-byte swizzle as written by TMA)
    const int m = ct >> 2, j = ct & 3, sw = (m >> 1) & 3;
    const float4 x = *reinterpret_cast<const float4*>(st32 + m * 64 + 16 * (j ^ sw));
    uint2 o[3];
    split4<NP>(x, o);
    const int off = m * 64 + 16 * ((2 * h + (j >> 1)) ^ sw) + 8 * (j & 1);
#pragma unroll
    for (int p = 0; p < NP; ++p) *reinterpret_cast<uint2*>(pst + p * A_TILE + off) = o[p];
  }
  {  // B: FP32 rows k of BN values (plain); column n becomes row n of B^T
    const int n = ct & (BN - 1), c = ct / BN, sw = (n >> 1) & 3;
    const float* b32 = reinterpret_cast<const float*>(st32 + A32_TILE);
    float e[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) e[k] = b32[(8 * c + k) * BN + n];
    uint4 o[3];
    split8<NP>(e, o);
    uint8_t* bt = pst + NP * A_TILE + n * 64 + 16 * ((2 * h + c) ^ sw);
#pragma unroll
    for (int p = 0; p < NP; ++p) *reinterpret_cast<uint4*>(bt + p * B_TILE) = o[p];
  }
}

// D64 epilogue: the FP64 combination of Sec. II-D for 16 columns of one row
// (chunk c), each partial product read from its own accumulator.
template <int MODE, int BN>
__device__ __forceinline__ void sum_products_f64(uint32_t tb, int c, double (&z)[16]) {
  float u[16], w[16];
  auto ld = [&](int a, int b, float (&v)[16]) {
    tmem_ld16_wait(tb + static_cast<uint32_t>(prod_slot(MODE, a, b) * BN + c * 16), v);
  };
  bool has = false;  // z holds the sum of the smaller levels
  auto add_level = [&](const double (&lv)[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = has ? lv[i] + z[i] : lv[i];
    has = true;
  };
  double lv[16];
  if constexpr (MODE == 9) {  // Z4 = Z22
    ld(2, 2, u);
#pragma unroll
    for (int i = 0; i < 16; ++i) lv[i] = widen(u[i]);
    add_level(lv);
  }
  if constexpr (MODE >= 8) {  // Z3 = Z12 + Z21
    ld(1, 2, u);
    ld(2, 1, w);
#pragma unroll
    for (int i = 0; i < 16; ++i) lv[i] = widen(u[i]) + widen(w[i]);
    add_level(lv);
  }
  if constexpr (MODE >= 6) {  // Z2 = Z02 + (Z11 + Z20)
    ld(1, 1, u);
    ld(2, 0, w);
#pragma unroll
    for (int i = 0; i < 16; ++i) lv[i] = widen(u[i]) + widen(w[i]);
    ld(0, 2, u);
#pragma unroll
    for (int i = 0; i < 16; ++i) lv[i] = widen(u[i]) + lv[i];
    add_level(lv);
  }
  if constexpr (MODE == 5) {  // Z2 = Z02 + Z11 (A has no third piece)
    ld(0, 2, u);
    ld(1, 1, w);
#pragma unroll
    for (int i = 0; i < 16; ++i) lv[i] = widen(u[i]) + widen(w[i]);
    add_level(lv);
  }
  if constexpr (MODE >= 3) {  // Z1 = Z01 + Z10
    ld(0, 1, u);
    ld(1, 0, w);
#pragma unroll
    for (int i = 0; i < 16; ++i) lv[i] = widen(u[i]) + widen(w[i]);
    add_level(lv);
  }
  ld(0, 0, u);  // Z = Z0 + (...)
#pragma unroll
  for (int i = 0; i < 16; ++i) lv[i] = widen(u[i]);
  add_level(lv);
}

template <int MODE, int BN, int BK, int STAGES, bool GROUPED, bool FUSED = false, bool D64 = false,
          int CH = 0>
__global__ void __launch_bounds__(TcConfig<MODE, BN, BK, STAGES, FUSED, D64, CH>::THREADS, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcArgs args) {
  using Cfg = TcConfig<MODE, BN, BK, STAGES, FUSED, D64, CH>;
  static_assert(!(D64 && GROUPED), "FP64 collection: single problem");
  constexpr uint32_t IDESC = idesc_bf16_f32<BM, BN>();
  // launched as a programmatic dependent of the previous kernel (the LU's
  // next-column update): wait for it to complete; a no-op otherwise
  asm volatile("griddepcontrol.wait;" ::: "memory");

  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw_addr = smem_addr(smem_raw);
  uint8_t* smem = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
  uint8_t* smem32 = smem + STAGES * Cfg::STAGE;  // fused: FP32 stages
  uint64_t* full = reinterpret_cast<uint64_t*>(smem32 + Cfg::S32 * Cfg::STAGE32);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + Cfg::ACC_BUFS;
  uint64_t* drain = acc_empty + Cfg::ACC_BUFS;
  uint64_t* full32 = drain + 1;  // fused only
  uint64_t* empty32 = full32 + Cfg::S32;
  uint64_t* chunk_full = empty32 + Cfg::S32;  // chunked only: a D_main buffer is complete
  uint64_t* chunk_empty = chunk_full + 2;     // ... and has been read
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(chunk_empty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* err = args.err;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      // fused: the piece stage is filled by the converter warps
      mbar_init(&full[s], FUSED ? Cfg::CONV_WARPS : 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < Cfg::S32; ++s) {
      mbar_init(&full32[s], 1);
      mbar_init(&empty32[s], Cfg::CONV_WARPS);
    }
    for (int b = 0; b < Cfg::ACC_BUFS; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 32 * Cfg::EPI_WARPS);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&chunk_full[b], 1);
      mbar_init(&chunk_empty[b], 32 * Cfg::EPI_WARPS);
    }
    mbar_init(drain, 1);
    fence_barrier_init();
    fence_proxy_async_smem();
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, Cfg::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------ TMA producer
      constexpr int NS = FUSED ? Cfg::S32 : STAGES;
      uint64_t* fbar = FUSED ? full32 : full;
      uint64_t* ebar = FUSED ? empty32 : empty;
      int s = 0;
      uint32_t ph = 0;
      int64_t issued = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < args.num_tiles && ok; t += gridDim.x) {
        const TileInfo ti = get_tile<GROUPED>(t, args);
        const int loads = FUSED ? 2 * ti.k_tiles : ti.k_tiles;
        for (int kt = 0; kt < loads; ++kt) {
          if (!mbar_wait_bounded(&ebar[s], ph ^ 1u, err, kErrWaitEmpty)) {
            ok = false;
            break;
          }
          if constexpr (FUSED) {
            // FP32 K-columns kt*16 .. kt*16+15 of the A row block and the B column block
            uint8_t* st = smem32 + s * Cfg::STAGE32;
            mbar_arrive_expect_tx(&fbar[s], Cfg::STAGE32);
            tma_load_2d(st, &tmA, &fbar[s], kt * Cfg::KF, ti.mb * BM);
            tma_load_2d(st + Cfg::A32_TILE, &tmB, &fbar[s], ti.nb * BN, kt * Cfg::KF);
          } else {
            uint8_t* st = smem + s * Cfg::STAGE;
            mbar_arrive_expect_tx(&fbar[s], Cfg::STAGE);
            tma_load_3d(st, &tmA, &fbar[s], kt * BK, ti.mb * BM, ti.c2);
            tma_load_3d(st + Cfg::STAGE_A, &tmB, &fbar[s], kt * BK, ti.nb * BN, ti.c2);
          }
          ++issued;
          if (++s == NS) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      // Every issued load must have landed before the CTA may exit: wait for
      // the last phase issued on each stage (already complete in normal runs).
      for (int q = 0; q < NS; ++q) {
        if (issued <= q) break;
        const int64_t last = q + ((issued - 1 - q) / NS) * NS;
        mbar_wait_bounded(&fbar[q], static_cast<uint32_t>((last / NS) & 1), err, kErrWaitDrain);
      }
    }
  } else if (FUSED && warp >= 6) {
    // -------------------------------------------------- converters (fused)
    const int ct = threadIdx.x - 192;  // 0..511
    int s32 = 0, sp = 0;
    uint32_t ph32 = 0, php = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < args.num_tiles && ok; t += gridDim.x) {
      const int k_tiles = get_tile<GROUPED>(t, args).k_tiles;
      for (int kt = 0; kt < k_tiles && ok; ++kt) {
        // the piece stage must have been consumed by the MMAs issued from it
        ok = mbar_wait_bounded(&empty[sp], php ^ 1u, err, kErrWaitEmpty);
        ok = __all_sync(0xFFFFFFFFu, ok);
        if (!ok) break;
        uint8_t* pst = smem + sp * Cfg::STAGE;
        for (int h = 0; h < 2; ++h) {
          ok = mbar_wait_bounded(&full32[s32], ph32, err, kErrWaitFull);
          ok = __all_sync(0xFFFFFFFFu, ok);
          if (!ok) break;
          convert_half<Cfg::NP, BN>(smem32 + s32 * Cfg::STAGE32, pst, h, ct);
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty32[s32]);  // FP32 stage free for the next load
          if (++s32 == Cfg::S32) {
            s32 = 0;
            ph32 ^= 1u;
          }
        }
        if (!ok) break;
        fence_proxy_async_smem();  // piece writes visible to the tensor core
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[sp]);
        if (++sp == STAGES) {
          sp = 0;
          php ^= 1u;
        }
      }
    }
  } else if (CH > 0 && warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------ MMA issuer (chunked)
      // hi*hi goes to D_main, restarted at every chunk of CH K-slices; the
      // corrections accumulate in D_corr over the whole K.  A chunk's first
      // hi*hi MMA waits until the epilogue has read the previous chunk's
      // D_main; the corrections of that K-slice, issued before it, keep the
      // tensor core busy meanwhile.
      int s = 0, gch = 0;
      uint32_t ph = 0, aph = 0;
      bool ok = true;
      const uint32_t dm = tmem_base;
      const uint32_t dc = tmem_base + static_cast<uint32_t>(BN);
      for (int t = blockIdx.x; t < args.num_tiles && ok; t += gridDim.x) {
        if (!mbar_wait_bounded(&acc_empty[0], aph ^ 1u, err, kErrWaitAccEmpty)) break;
        tc_fence_after();
        const int k_tiles = get_tile<GROUPED>(t, args).k_tiles;
        for (int kt = 0; kt < k_tiles && ok; ++kt) {
          const int kc = kt % CH;
          if (!mbar_wait_bounded(&full[s], ph, err, kErrWaitFull)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_addr(smem + s * Cfg::STAGE);
          const uint32_t sb = sa + Cfg::STAGE_A;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
            for (int p = 0; p < Cfg::NPROD; ++p) {
              const Prod pr = prod_of(MODE, p);
              const uint64_t ad = smem_desc_kmajor<Cfg::SW>(sa + pr.a * Cfg::A_TILE + kk * 32);
              const uint64_t bd = smem_desc_kmajor<Cfg::SW>(sb + pr.b * Cfg::B_TILE + kk * 32);
              if (pr.acc == 0) {
                if (kc == 0 && kk == 0 && gch > 0) {  // D_main of chunk gch-1 read?
                  if (!mbar_wait_bounded(&chunk_empty[0], (gch - 1) & 1, err, kErrWaitAccEmpty)) {
                    ok = false;
                    break;
                  }
                  tc_fence_after();
                }
                umma_bf16_ss(dm, ad, bd, IDESC, (kc > 0 || kk > 0) ? 1u : 0u);
              } else {
                umma_bf16_ss(dc, ad, bd, IDESC,
                             (kt > 0 || kk > 0 || !first_in_acc(MODE, p)) ? 1u : 0u);
              }
            }
            if (!ok) break;
          }
          if (!ok) break;
          umma_commit(&empty[s]);
          if (++s == STAGES) {
            s = 0;
            ph ^= 1u;
          }
          if (kc == CH - 1 || kt == k_tiles - 1) {
            umma_commit(&chunk_full[0]);
            ++gch;
          }
        }
        if (!ok) break;
        umma_commit(&acc_full[0]);
        aph ^= 1u;
      }
      umma_commit(drain);
      mbar_wait_bounded(drain, 0u, err, kErrWaitDrain);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------ MMA issuer
      int s = 0, buf = 0;
      uint32_t ph = 0, aph = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < args.num_tiles && ok; t += gridDim.x) {
        if (!mbar_wait_bounded(&acc_empty[buf], aph ^ 1u, err, kErrWaitAccEmpty)) break;
        tc_fence_after();
        const uint32_t d0 = tmem_base + static_cast<uint32_t>(buf * Cfg::NACC * BN);
        const int k_tiles = get_tile<GROUPED>(t, args).k_tiles;
        for (int kt = 0; kt < k_tiles; ++kt) {
          if (!mbar_wait_bounded(&full[s], ph, err, kErrWaitFull)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_addr(smem + s * Cfg::STAGE);
          const uint32_t sb = sa + Cfg::STAGE_A;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
            for (int p = 0; p < Cfg::NPROD; ++p) {
              const Prod pr = prod_of(MODE, p);
              const uint64_t ad = smem_desc_kmajor<Cfg::SW>(sa + pr.a * Cfg::A_TILE + kk * 32);
              const uint64_t bd = smem_desc_kmajor<Cfg::SW>(sb + pr.b * Cfg::B_TILE + kk * 32);
              const uint32_t accum =
                  (kt > 0 || kk > 0 || (!D64 && !first_in_acc(MODE, p))) ? 1u : 0u;
              umma_bf16_ss(d0 + static_cast<uint32_t>((D64 ? p : pr.acc) * BN), ad, bd, IDESC,
                           accum);
            }
          }
          umma_commit(&empty[s]);
          if (++s == STAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(&acc_full[buf]);
        if (++buf == Cfg::ACC_BUFS) {
          buf = 0;
          aph ^= 1u;
        }
      }
      // all MMAs issued by this thread complete before tensor memory is freed
      umma_commit(drain);
      mbar_wait_bounded(drain, 0u, err, kErrWaitDrain);
    }
  } else if constexpr (CH > 0) {
    // -------------------------------------------------- epilogue (chunked)
    // Each chunk's D_main is added into S in FP32 with round to nearest (a
    // thread holds a quarter of its row's BN values: warps 2..5 the first
    // quarter, 6..9 the second, ...), then Z = S + D_corr.
    constexpr int HB = BN / (Cfg::EPI_WARPS / 4);  // columns a thread holds
    static_assert(HB % 16 == 0, "half tile in groups of 16 columns");
    const int q = warp & 3;
    const int row_in_tile = q * 32 + lane;
    const int hc = ((warp - 2) >> 2) * HB;  // first column of this thread's part
    const uint32_t lane_off = (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(hc);
    int gce = 0;
    uint32_t aph = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < args.num_tiles && ok; t += gridDim.x) {
      const TileInfo ti = get_tile<GROUPED>(t, args);
      const int nch = (ti.k_tiles + CH - 1) / CH;
      float S[HB];
      for (int ch = 0; ch < nch; ++ch) {
        ok = mbar_wait_bounded(&chunk_full[0], gce & 1, err, kErrWaitAccFull);
        ok = __all_sync(0xFFFFFFFFu, ok);
        if (!ok) break;
        tc_fence_after();
        const uint32_t tb = tmem_base + lane_off;
#pragma unroll
        for (int c = 0; c < HB / 16; ++c) {
          float v[16];
          tmem_ld16_wait(tb + c * 16, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) S[c * 16 + i] = ch == 0 ? v[i] : S[c * 16 + i] + v[i];
        }
        tc_fence_before();
        mbar_arrive(&chunk_empty[0]);
        ++gce;
      }
      if (!ok) break;
      ok = mbar_wait_bounded(&acc_full[0], aph, err, kErrWaitAccFull);
      ok = __all_sync(0xFFFFFFFFu, ok);
      if (!ok) break;
      tc_fence_after();
      // Z = D_main + D_corr, written over D_corr, then stored from there
      const uint32_t tdc = tmem_base + lane_off + static_cast<uint32_t>(BN);
#pragma unroll
      for (int c = 0; c < HB / 16; ++c) {
        float v[16];
        tmem_ld16_wait(tdc + c * 16, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = S[c * 16 + i] + v[i];
        tmem_st16_wait(tdc + c * 16, v);
      }
      const int row = ti.mb * BM + row_in_tile;
      const bool row_ok = row < ti.M;
      float* crow = ti.C + static_cast<int64_t>(row_ok ? row : 0) * ti.ldc;
#pragma unroll 1
      for (int c = 0; c < HB / 16; ++c) {
        float v[16];
        tmem_ld16_wait(tdc + c * 16, v);
        if (c == HB / 16 - 1) {
          tc_fence_before();
          mbar_arrive(&acc_empty[0]);
        }
        if (!row_ok) continue;
        const int col0 = ti.nb * BN + hc + c * 16;
        if (col0 >= ti.N) continue;
        float* dst = crow + col0;
        if (ti.vec_c && col0 + 16 <= ti.N) {
#pragma unroll
          for (int i = 0; i < 16; i += 4) {
            float4 o;
            float4 old = make_float4(0.f, 0.f, 0.f, 0.f);
            if (args.beta != 0.0f) old = *reinterpret_cast<const float4*>(dst + i);
            o.x = args.alpha * v[i + 0];
            o.y = args.alpha * v[i + 1];
            o.z = args.alpha * v[i + 2];
            o.w = args.alpha * v[i + 3];
            if (args.beta != 0.0f) {
              o.x = fmaf(args.beta, old.x, o.x);
              o.y = fmaf(args.beta, old.y, o.y);
              o.z = fmaf(args.beta, old.z, o.z);
              o.w = fmaf(args.beta, old.w, o.w);
            }
            *reinterpret_cast<float4*>(dst + i) = o;
          }
        } else {
          const int lim = min(16, ti.N - col0);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            if (i < lim) {
              const float tv = args.alpha * v[i];
              dst[i] = (args.beta == 0.0f) ? tv : fmaf(args.beta, dst[i], tv);
            }
          }
        }
      }
      aph ^= 1u;
    }
  } else {
    // -------------------------------------------------- epilogue (warps 2..5)
    const int q = warp & 3;  // tensor-memory lane quarter this warp may access
    const int row_in_tile = q * 32 + lane;
    int buf = 0;
    uint32_t aph = 0;
    for (int t = blockIdx.x; t < args.num_tiles; t += gridDim.x) {
      const TileInfo ti = get_tile<GROUPED>(t, args);
      const int mb = ti.mb, nb = ti.nb;
      const int row = mb * BM + row_in_tile;
      const bool row_ok = row < ti.M;
      // With beta != 0 and a narrow tile, the tile's C row is loaded before
      // the accumulator is awaited, so its latency overlaps the MMAs (the
      // short-K trailing updates of the batched LU spent their time in these
      // loads, one 16-column piece after another).
      constexpr int PFC = (!D64 && BN <= 64) ? BN / 16 : 0;
      float cpre[PFC > 0 ? PFC : 1][16];
      const bool pre = PFC > 0 && args.beta != 0.0f && row_ok;
      if constexpr (PFC > 0) {
        if (pre) {
          const float* src = ti.C + static_cast<int64_t>(row) * ti.ldc;
#pragma unroll
          for (int c = 0; c < PFC; ++c) {
            const int col0 = nb * BN + c * 16;
#pragma unroll
            for (int i = 0; i < 16; ++i) cpre[c][i] = col0 + i < ti.N ? src[col0 + i] : 0.0f;
          }
        }
      }
      bool ok = mbar_wait_bounded(&acc_full[buf], aph, err, kErrWaitAccFull);
      ok = __all_sync(0xFFFFFFFFu, ok);
      if (!ok) break;
      tc_fence_after();
      const uint32_t tb = tmem_base + (static_cast<uint32_t>(q * 32) << 16) +
                          static_cast<uint32_t>(buf * Cfg::NACC * BN);
      if constexpr (D64) {
        double* drow = args.Cd + static_cast<int64_t>(row_ok ? row : 0) * args.ldc;
#pragma unroll 1
        for (int c = 0; c < BN / 16; ++c) {
          __syncwarp();
          double z[16];
          sum_products_f64<MODE, BN>(tb, c, z);
          if (c == BN / 16 - 1) {
            tc_fence_before();
            mbar_arrive(&acc_empty[buf]);
          }
          if (!row_ok) continue;
          const int col0 = nb * BN + c * 16;
          if (col0 >= ti.N) continue;
          double* dst = drow + col0;
          if (args.vec_c && col0 + 16 <= ti.N) {
#pragma unroll
            for (int i = 0; i < 16; i += 2)
              *reinterpret_cast<double2*>(dst + i) = make_double2(z[i], z[i + 1]);
          } else {
            const int lim = min(16, ti.N - col0);
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (i < lim) dst[i] = z[i];
          }
        }
        if (++buf == Cfg::ACC_BUFS) {
          buf = 0;
          aph ^= 1u;
        }
        continue;
      }
      float* crow = ti.C + static_cast<int64_t>(row_ok ? row : 0) * ti.ldc;
#pragma unroll(PFC > 0 ? PFC : 1)
      for (int c = 0; c < BN / 16; ++c) {
        __syncwarp();
        float v[16];
        tmem_ld16_wait(tb + c * 16, v);
        if (Cfg::NACC == 2) {
          float w[16];
          tmem_ld16_wait(tb + BN + c * 16, w);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = v[i] + w[i];  // Z = D_main + D_corr
        }
        if (c == BN / 16 - 1) {
          tc_fence_before();
          mbar_arrive(&acc_empty[buf]);
        }
        if (!row_ok) continue;
        const int col0 = nb * BN + c * 16;
        if (col0 >= ti.N) continue;
        float* dst = crow + col0;
        if (ti.vec_c && col0 + 16 <= ti.N) {
#pragma unroll
          for (int i = 0; i < 16; i += 4) {
            float4 o;
            float4 old = make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (PFC > 0) {
              if (pre) old = make_float4(cpre[c][i], cpre[c][i + 1], cpre[c][i + 2], cpre[c][i + 3]);
              else if (args.beta != 0.0f) old = *reinterpret_cast<const float4*>(dst + i);
            } else {
              if (args.beta != 0.0f) old = *reinterpret_cast<const float4*>(dst + i);
            }
            o.x = args.alpha * v[i + 0];
            o.y = args.alpha * v[i + 1];
            o.z = args.alpha * v[i + 2];
            o.w = args.alpha * v[i + 3];
            if (args.beta != 0.0f) {
              o.x = fmaf(args.beta, old.x, o.x);
              o.y = fmaf(args.beta, old.y, o.y);
              o.z = fmaf(args.beta, old.z, o.z);
              o.w = fmaf(args.beta, old.w, o.w);
            }
            *reinterpret_cast<float4*>(dst + i) = o;
          }
        } else {
          const int lim = min(16, ti.N - col0);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            if (i < lim) {
              const float tv = args.alpha * v[i];
              float cv = 0.0f;
              if constexpr (PFC > 0) {
                if (args.beta != 0.0f) cv = pre ? cpre[c][i] : dst[i];
              } else {
                if (args.beta != 0.0f) cv = dst[i];
              }
              dst[i] = (args.beta == 0.0f) ? tv : fmaf(args.beta, cv, tv);
            }
          }
        }
      }
      if (++buf == Cfg::ACC_BUFS) {
        buf = 0;
        aph ^= 1u;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem_base, Cfg::TMEM_COLS);
  }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  // function-local static: initialised once, thread-safe
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
  }();
  return fn;
}

// 3-D bfloat16 tensor {inner (K), rows, planes}, box {bk, box_rows, box_planes}
// (box_planes = all planes by default).
bool make_piece_map(CUtensorMap* map, const uint16_t* base, int64_t inner, int64_t rows,
                    int planes, int64_t ld, int64_t plane, int bk, int box_rows,
                    int box_planes = 0) {
  auto fn = encode_fn();
  if (!fn) return false;
  // the driver-API encoder needs a current context on this thread; make the
  // current device's primary context current (a no-op if it already is)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) return false;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(rows),
                        static_cast<cuuint64_t>(planes)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(ld) * 2, static_cast<cuuint64_t>(plane) * 2};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(bk), static_cast<cuuint32_t>(box_rows),
                       static_cast<cuuint32_t>(box_planes > 0 ? box_planes : planes)};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapSwizzle sw = (bk * 2 == 128) ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(base), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C: float* (FP32 result, alpha/beta applied) or, with D64, double* (the
// FP64 collection, alpha/beta unused).
template <int MODE, int BN, int BK, int STAGES, bool D64 = false, int CH = 0>
bfx_status run_tc(int64_t m, int64_t n, int64_t k, float alpha, const uint16_t* Ap, int64_t lda_p,
                  int64_t a_plane, const uint16_t* Btp, int64_t ldb_p, int64_t b_plane,
                  float beta, void* C, int64_t ldc, cudaStream_t s, bool pdl = false) {
  using Cfg = TcConfig<MODE, BN, BK, STAGES, false, D64, CH>;
  // with a single piece only plane 0 is read; any legal plane stride will do
  if (Cfg::NPA == 1) a_plane = round_up(lda_p * m, 8);
  if (Cfg::NPB == 1) b_plane = round_up(ldb_p * n, 8);
  CUtensorMap ma, mb;
  if (!make_piece_map(&ma, Ap, k, m, Cfg::NPA, lda_p, a_plane, BK, BM)) return BFX_EUNSUPPORTED;
  if (!make_piece_map(&mb, Btp, k, n, Cfg::NPB, ldb_p, b_plane, BK, BN)) return BFX_EUNSUPPORTED;
  TcArgs a;
  a.M = static_cast<int>(m);
  a.N = static_cast<int>(n);
  a.K = static_cast<int>(k);
  a.tiles_m = static_cast<int>(ceil_div(m, BM));
  a.tiles_n = static_cast<int>(ceil_div(n, BN));
  const int64_t tiles = static_cast<int64_t>(a.tiles_m) * a.tiles_n;
  if (tiles > INT32_MAX) return BFX_EUNSUPPORTED;
  a.num_tiles = static_cast<int>(tiles);
  a.k_tiles = static_cast<int>(ceil_div(k, BK));
  a.alpha = alpha;
  a.beta = beta;
  a.C = D64 ? nullptr : static_cast<float*>(C);
  a.Cd = D64 ? static_cast<double*>(C) : nullptr;
  a.ldc = ldc;
  a.vec_c = (ldc % (D64 ? 2 : 4) == 0) && aligned(C, 16);
  a.err = device_error_word();
  a.tiles = nullptr;
  a.probs = nullptr;
  if (!a.err) return BFX_ECUDA;
  auto kern = gemm_tc_kernel<MODE, BN, BK, STAGES, false, false, D64, CH>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM) !=
      cudaSuccess)
    return BFX_ECUDA;
  const int sms = current_num_sms();
  const int grid = static_cast<int>(tiles < sms ? tiles : sms);
  if (pdl) {  // may start while the previous kernel on s finishes (the kernel waits for it)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(Cfg::THREADS);
    cfg.dynamicSmemBytes = Cfg::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, ma, mb, a) != cudaSuccess) return BFX_ECUDA;
    return BFX_OK;
  }
  kern<<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(ma, mb, a);
  return last_launch_status();
}

// 2-D FP32 tensor {inner, rows} with row stride ld elements, box {box_inner, box_rows}.
bool make_f32_map(CUtensorMap* map, const float* base, int64_t inner, int64_t rows, int64_t ld,
                  int box_inner, int box_rows, CUtensorMapSwizzle sw) {
  auto fn = encode_fn();
  if (!fn) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 4};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_inner), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE, int STAGES>
bfx_status run_tc_fused(int64_t m, int64_t n, int64_t k, float alpha, const float* A, int64_t lda,
                        const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                        cudaStream_t s) {
  constexpr int BN = 256, BK = 32;
  using Cfg = TcConfig<MODE, BN, BK, STAGES, true>;
  CUtensorMap ma, mb;
  if (!make_f32_map(&ma, A, k, m, lda, Cfg::KF, BM, CU_TENSOR_MAP_SWIZZLE_64B))
    return BFX_EUNSUPPORTED;
  if (!make_f32_map(&mb, B, n, k, ldb, BN, Cfg::KF, CU_TENSOR_MAP_SWIZZLE_NONE))
    return BFX_EUNSUPPORTED;
  TcArgs a{};
  a.M = static_cast<int>(m);
  a.N = static_cast<int>(n);
  a.K = static_cast<int>(k);
  a.tiles_m = static_cast<int>(ceil_div(m, BM));
  a.tiles_n = static_cast<int>(ceil_div(n, BN));
  const int64_t tiles = static_cast<int64_t>(a.tiles_m) * a.tiles_n;
  if (tiles > INT32_MAX) return BFX_EUNSUPPORTED;
  a.num_tiles = static_cast<int>(tiles);
  a.k_tiles = static_cast<int>(ceil_div(k, BK));
  a.alpha = alpha;
  a.beta = beta;
  a.C = C;
  a.ldc = ldc;
  a.vec_c = (ldc % 4 == 0) && aligned(C, 16);
  a.err = device_error_word();
  if (!a.err) return BFX_ECUDA;
  auto kern = gemm_tc_kernel<MODE, BN, BK, STAGES, false, true>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM) !=
      cudaSuccess)
    return BFX_ECUDA;
  const int sms = current_num_sms();
  const int grid = static_cast<int>(tiles < sms ? tiles : sms);
  kern<<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(ma, mb, a);
  return last_launch_status();
}

template <int MODE, int BN, int BK, int STAGES>
bfx_status run_tc_grouped(int num_tiles, const GroupTile* d_tiles, const GroupProblem* d_probs,
                          const uint16_t* Apack, int64_t a_rows, const uint16_t* Bpack,
                          int64_t b_rows, int64_t planes, int64_t kp, float alpha, float beta,
                          cudaStream_t s) {
  using Cfg = TcConfig<MODE, BN, BK, STAGES>;
  CUtensorMap ma, mb;
  static_assert(Cfg::NPA == Cfg::NPB, "grouped: symmetric modes");
  if (!make_piece_map(&ma, Apack, kp, a_rows, static_cast<int>(planes), kp, a_rows * kp, BK, BM,
                      Cfg::NPA))
    return BFX_EUNSUPPORTED;
  if (!make_piece_map(&mb, Bpack, kp, b_rows, static_cast<int>(planes), kp, b_rows * kp, BK, BN,
                      Cfg::NPB))
    return BFX_EUNSUPPORTED;
  TcArgs a{};
  a.num_tiles = num_tiles;
  a.alpha = alpha;
  a.beta = beta;
  a.err = device_error_word();
  a.tiles = d_tiles;
  a.probs = d_probs;
  if (!a.err) return BFX_ECUDA;
  auto kern = gemm_tc_kernel<MODE, BN, BK, STAGES, true>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM) !=
      cudaSuccess)
    return BFX_ECUDA;
  const int sms = current_num_sms();
  const int grid = num_tiles < sms ? num_tiles : sms;
  kern<<<grid, 192, Cfg::SMEM, s>>>(ma, mb, a);
  return last_launch_status();
}

}  // namespace

int gemm_bk(bfx_mode mode) { return mode == BFX_X1 ? 64 : 32; }

// Grouped launches for one UMMA N (tile width of the grouped problems).
template <int BN>
bfx_status grouped_bn(bfx_mode mode, int num_tiles, const GroupTile* d_tiles,
                      const GroupProblem* d_probs, const uint16_t* Apack, int64_t a_rows,
                      const uint16_t* Bpack, int64_t b_rows, int64_t planes, int64_t kp,
                      float alpha, float beta, cudaStream_t s) {
  // stages: as many as fit (at most 6); a narrower tile holds more in flight
  constexpr int S1 = BN == 256 ? 4 : 6, S3 = BN == 256 ? 4 : 6, S6 = BN == 256 ? 3 : (BN == 128 ? 4 : 5);
  switch (mode) {
    case BFX_X1:
      return run_tc_grouped<1, BN, 64, S1>(num_tiles, d_tiles, d_probs, Apack, a_rows, Bpack,
                                           b_rows, planes, kp, alpha, beta, s);
    case BFX_X3:
      return run_tc_grouped<3, BN, 32, S3>(num_tiles, d_tiles, d_probs, Apack, a_rows, Bpack,
                                           b_rows, planes, kp, alpha, beta, s);
    case BFX_X6:
      return run_tc_grouped<6, BN, 32, S6>(num_tiles, d_tiles, d_probs, Apack, a_rows, Bpack,
                                           b_rows, planes, kp, alpha, beta, s);
    case BFX_X8:
      return run_tc_grouped<8, BN, 32, S6>(num_tiles, d_tiles, d_probs, Apack, a_rows, Bpack,
                                           b_rows, planes, kp, alpha, beta, s);
    case BFX_X9:
      return run_tc_grouped<9, BN, 32, S6>(num_tiles, d_tiles, d_probs, Apack, a_rows, Bpack,
                                           b_rows, planes, kp, alpha, beta, s);
    default:
      return BFX_EINVAL;
  }
}

bfx_status launch_gemm_grouped(bfx_mode mode, int bn, int num_tiles, const GroupTile* d_tiles,
                               const GroupProblem* d_probs, const uint16_t* Apack,
                               int64_t a_rows, const uint16_t* Bpack, int64_t b_rows,
                               int64_t planes, int64_t kp, float alpha, float beta,
                               cudaStream_t s) {
  if (num_tiles <= 0) return BFX_OK;
  switch (bn) {
    case 64:
      return grouped_bn<64>(mode, num_tiles, d_tiles, d_probs, Apack, a_rows, Bpack, b_rows,
                            planes, kp, alpha, beta, s);
    case 128:
      return grouped_bn<128>(mode, num_tiles, d_tiles, d_probs, Apack, a_rows, Bpack, b_rows,
                             planes, kp, alpha, beta, s);
    case 256:
      return grouped_bn<256>(mode, num_tiles, d_tiles, d_probs, Apack, a_rows, Bpack, b_rows,
                             planes, kp, alpha, beta, s);
    default:
      return BFX_EINVAL;
  }
}

bfx_status launch_gemm_fused(bfx_mode mode, int64_t m, int64_t n, int64_t k, float alpha,
                             const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                             float* C, int64_t ldc, cudaStream_t s) {
  if (m == 0 || n == 0) return BFX_OK;
  if (k == 0) return launch_scale(m, n, beta, C, ldc, s);
  // TMA: 16-byte aligned bases and row strides
  if (lda % 4 != 0 || ldb % 4 != 0 || !aligned(A, 16) || !aligned(B, 16)) return BFX_EUNSUPPORTED;
  switch (mode) {
    case BFX_X1:
      return run_tc_fused<1, 2>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
    case BFX_X3:
      return run_tc_fused<3, 2>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
    case BFX_X6:
      return run_tc_fused<6, 2>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
    case BFX_X8:
      return run_tc_fused<8, 2>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
    case BFX_X9:
      return run_tc_fused<9, 2>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
    default:
      return BFX_EINVAL;
  }
}

bfx_status launch_gemm_presplit(bfx_mode mode, int64_t m, int64_t n, int64_t k, float alpha,
                                const uint16_t* Ap, int64_t lda_p, int64_t a_plane,
                                const uint16_t* Btp, int64_t ldb_p, int64_t b_plane, float beta,
                                float* C, int64_t ldc, cudaStream_t s, bool pdl) {
  if (m == 0 || n == 0) return BFX_OK;
  if (k == 0) return launch_scale(m, n, beta, C, ldc, s);
  if (k > kChunkMinK) {
    // long K, FP32-accurate modes: hi*hi accumulated in chunks of kChunkK,
    // the chunk sums added with round to nearest by the epilogue.  x3 and x5
    // keep one accumulator: their error is that of the dropped 2^-16 terms.
    switch (mode) {
      case BFX_X6:
        return run_tc<6, 256, 32, 3, false, kChunkK / 32>(m, n, k, alpha, Ap, lda_p, a_plane, Btp,
                                                          ldb_p, b_plane, beta, C, ldc, s, pdl);
      case BFX_X8:
        return run_tc<8, 256, 32, 3, false, kChunkK / 32>(m, n, k, alpha, Ap, lda_p, a_plane, Btp,
                                                          ldb_p, b_plane, beta, C, ldc, s, pdl);
      case BFX_X9:
        return run_tc<9, 256, 32, 3, false, kChunkK / 32>(m, n, k, alpha, Ap, lda_p, a_plane, Btp,
                                                          ldb_p, b_plane, beta, C, ldc, s, pdl);
      default:
        break;
    }
  }
  switch (mode) {
    case BFX_X1:
      return run_tc<1, 256, 64, 4>(m, n, k, alpha, Ap, lda_p, a_plane, Btp, ldb_p, b_plane, beta,
                                   C, ldc, s, pdl);
    case BFX_X3:
      return run_tc<3, 256, 32, 4>(m, n, k, alpha, Ap, lda_p, a_plane, Btp, ldb_p, b_plane, beta,
                                   C, ldc, s, pdl);
    case BFX_X5:
      return run_tc<5, 256, 32, 3>(m, n, k, alpha, Ap, lda_p, a_plane, Btp, ldb_p, b_plane, beta,
                                   C, ldc, s, pdl);
    case BFX_X6:
      return run_tc<6, 256, 32, 3>(m, n, k, alpha, Ap, lda_p, a_plane, Btp, ldb_p, b_plane, beta,
                                   C, ldc, s, pdl);
    case BFX_X8:
      return run_tc<8, 256, 32, 3>(m, n, k, alpha, Ap, lda_p, a_plane, Btp, ldb_p, b_plane, beta,
                                   C, ldc, s, pdl);
    case BFX_X9:
      return run_tc<9, 256, 32, 3>(m, n, k, alpha, Ap, lda_p, a_plane, Btp, ldb_p, b_plane, beta,
                                   C, ldc, s, pdl);
    default:
      return BFX_EINVAL;
  }
}

// The FP64 collection ("d", Sec. IV-A): one accumulator per product, so the
// tile is 64 columns wide (32 for x9) to fit tensor memory's 512 columns.
bfx_status launch_gemm_f64(bfx_mode mode, int64_t m, int64_t n, int64_t k, const uint16_t* Ap,
                           int64_t lda_p, int64_t a_plane, const uint16_t* Btp, int64_t ldb_p,
                           int64_t b_plane, double* C, int64_t ldc, cudaStream_t s) {
  if (m == 0 || n == 0) return BFX_OK;
  switch (mode) {
    case BFX_X1:
      return run_tc<1, 64, 64, 6, true>(m, n, k, 1.f, Ap, lda_p, a_plane, Btp, ldb_p, b_plane,
                                        0.f, C, ldc, s);
    case BFX_X3:
      return run_tc<3, 64, 32, 6, true>(m, n, k, 1.f, Ap, lda_p, a_plane, Btp, ldb_p, b_plane,
                                        0.f, C, ldc, s);
    case BFX_X5:
      return run_tc<5, 64, 32, 6, true>(m, n, k, 1.f, Ap, lda_p, a_plane, Btp, ldb_p, b_plane,
                                        0.f, C, ldc, s);
    case BFX_X6:
      return run_tc<6, 64, 32, 5, true>(m, n, k, 1.f, Ap, lda_p, a_plane, Btp, ldb_p, b_plane,
                                        0.f, C, ldc, s);
    case BFX_X8:
      return run_tc<8, 64, 32, 5, true>(m, n, k, 1.f, Ap, lda_p, a_plane, Btp, ldb_p, b_plane,
                                        0.f, C, ldc, s);
    case BFX_X9:
      return run_tc<9, 32, 32, 6, true>(m, n, k, 1.f, Ap, lda_p, a_plane, Btp, ldb_p, b_plane,
                                        0.f, C, ldc, s);
    default:
      return BFX_EINVAL;
  }
}

}  // namespace bfx
