// legendre_tc.cu -- the mixed form's Legendre synthesis (Eq. syn2) with the
// contraction of a_lm against Lambda_lm on the tensor cores (tcgen05).
//
// For one m and the 128 ring pairs of a CTA the synthesis is a product
// F[pair][col] = sum_l Lambda[pair][l] B[l][col] (Sect. 3.2's inner loop over l,
// Fig. 1), with B the a_lm values arranged by column (real and imaginary parts,
// the even/odd-l split of the ring-pair parity, the +s / -s spin combinations).
// Lambda is still generated on the fly by the double-float recursion of Sect. 4.1
// (one thread per ring pair, as in legendre_mixed.cu); the product runs as bf16
// matrix products with FP32 accumulation, made exact by splitting both operands
// into digits on a common grid (an Ozaki-style error-free split):
//
//  * Lambda = L0 + L1 + L2 + r.  The digits Lj are multiples of qj = u 2^(-7-8j)
//    with |Lj| <= 128 qj, where u is a power of two bounding the ring pair's own
//    |Lambda_lm| from its join block to lmax + 1 (its join record: one walk of the
//    recursion at plan creation; not below 2^-16 of the plan-wide bound
//    sqrt((2 lmax + 3)/(4 pi)), |d^l| <= 1); each digit fits a bf16 exactly.  One
//    row of the product is one pair, so rows on different grids never share a sum.
//    The FP32 remainder r (|r| <= q2/2) is contracted on the CUDA cores (one FFMA
//    per output column), so Lambda enters to ~2^-43 u.
//  * B = B0 + ... + B5 with digits on the grid u_c 2^(-7-8j), u_c a power of two
//    bounding column c of B over a window of 256 degrees: a value enters to
//    2^-47 u_c (the last digit's rounding and that of the low word's entry; with
//    five digits the truncation at 2^-40 u_c was the larger error).
//  * The products Li Bj with i + j = k are accumulated in TMEM level k (k <= 5;
//    the dropped products sum to below 2^-47 of the bounds).  Every product is a
//    multiple of the level's quantum and a level's sum over one window stays
//    below 2^24 quanta, so the FP32 accumulation is exact whatever its rounding.
//  * After each window the six levels are read from TMEM and added in
//    double-float, together with the CUDA-core remainder sums.
//
// MMA shape: M = 128 ring pairs (one TMEM lane per pair: thread t reads lane t),
// K = 16 degrees per instruction, N = 2 NCW: one instruction reads two
// consecutive a_lm digit tiles (NCW >= 8 columns each) and so adds L_i B_j and
// L_i B_(j+1) into two consecutive levels of NCW TMEM columns (level k at column
// k NCW), which keeps the narrow shapes' MMAs free of padding columns: 8 MMAs per
// Lambda set and K-step instead of 14.
// A (the Lambda digits) and B (the a_lm digit stack) are K-major in shared memory
// without swizzle, 8x16-byte core matrices 128 bytes apart along K and 256 bytes
// apart along M / N.  One thread issues a K-step's MMAs in program order (the
// first ones of a window overwrite every level read later); the recursion's
// digits of K-step s + 1 are written once the MMAs of s have completed, and B is
// rebuilt then too.
#include "tcgen05.cuh"

namespace sht {
namespace tc {

constexpr int kRows = 128;          // ring pairs per CTA = MMA M = TMEM lanes
constexpr int kK = 16;              // degrees per MMA (bf16 K)
constexpr int kWin = 16;            // K-steps per TMEM window (256 degrees)
constexpr int kLamDigits = 3;       // bf16 digits of Lambda (plus an FP32 remainder)
constexpr int kAlmDigits = 6;       // bf16 digits of the a_lm columns
constexpr int kLevels = 6;          // TMEM levels read: digit products with i + j <= 5
constexpr int kATile = kRows * kK * 2;  // bytes of one 128 x 16 bf16 tile
constexpr int kPack = 4;            // degrees of digits held in registers before a shared-memory store
// the thread issuing the MMAs: lane 0 of the last warp, whose threads neither load
// the staged rows nor build B (threads 0-63 at one E/B pair), so that the warps
// reach the K-step's barrier together (152.4 -> 151.8 ms per headline pair)
constexpr int kIssuerThread = 96;
// Shapes: NCOL output columns per pair (spin: N1, S4, N2, S3 as re/im per job;
// spin 0: even-l and odd-l sums as re/im per job), NCW = max(NCOL, 8) TMEM columns
// per level and rows per a_lm digit tile, MMA width N = 2 NCW (two digit tiles, two
// levels), NV a_lm values per degree (spin: P = E + iB and M = E - iB, re and im;
// spin 0: re, im).  A set's digit stack holds the tiles of digits -1 .. 5, that of
// digit -1 zero: Lambda digit i meets the windows of digits
// (j0, j0 + 1) with j0 = -(i mod 2), j0 + 2, ..., which start on even levels i + j0,
// so every MMA writes the 2 NCW columns of a level pair at a multiple of N.
template <int NJ, bool SPIN>
struct Shape {
  static constexpr int NL = SPIN ? 2 : 1;
  static constexpr int NCOL = SPIN ? 8 * NJ : 4 * NJ;
  static constexpr int NCW = NCOL < 8 ? 8 : NCOL;
  static constexpr int N = 2 * NCW;
  static constexpr int NDT = kAlmDigits + 1;  // digit tiles per Lambda set: -1 .. 5
  static constexpr int COLS = kLevels * NCW;  // TMEM: levels 0 .. 5
  static constexpr int TCOLS = COLS <= 32 ? 32 : (COLS <= 64 ? 64 : (COLS <= 128 ? 128 : 256));
  static constexpr int NV = SPIN ? 4 * NJ : 2 * NJ;
  static constexpr int DTILE = NCW * kK * 2;  // bytes of one a_lm digit tile
  static constexpr int A_BYTES = NL * kLamDigits * kATile;
  static constexpr int B_BYTES = NL * NDT * DTILE;
  // per degree of a K-step, staged in shared memory one K-step ahead: the two
  // float4 of its recursion coefficients and one float4 per a_lm table row read
  static constexpr int NARR = SPIN ? 2 * NJ : NJ;
  static constexpr int ROW = 2 + NARR;
  static constexpr int STG = kK * ROW;                 // float4 per K-step
  static constexpr int PF = (STG + kRows - 1) / kRows;  // of them per thread
  static constexpr int ST_BYTES = 2 * STG * 16;        // two buffers
  static constexpr int ACC_BYTES = NCOL * kRows * 8;  // the double-float column sums [col][pair]
  static constexpr int SMEM = A_BYTES + ST_BYTES + B_BYTES + ACC_BYTES + 2 * NV * 4;
  // CTAs per SM the kernel is compiled for, and the dynamic shared memory
  // requested: at least enough that no more than 512 / TCOLS CTAs fit on an SM,
  // so their TMEM allocations never wait for one another
  static constexpr int MINB = TCOLS <= 64 ? 5 : (TCOLS == 128 ? 4 : 2);
  static constexpr int SMEM_FLOOR = (228 * 1024) / (512 / TCOLS + 1) - 1024 + 1;
  static constexpr int SMEM_LAUNCH = SMEM > SMEM_FLOOR ? SMEM : SMEM_FLOOR;
  static_assert(N % 16 == 0 && N <= 256 && NCW % 8 == 0, "MMA width; digit tiles of whole core-matrix rows");
  static_assert(kLevels % 2 == 0 && kLamDigits <= 3, "level pairs");
  static_assert(COLS <= TCOLS, "TMEM allocation");
  static_assert(NCOL <= 32, "tensor-core synthesis: at most 32 output columns");
  static_assert(128 % NV == 0, "a_lm values per degree must divide the CTA");
};



// the double-float a_lm value v (Shape::NV of them per degree) at table index ci
template <int NJ, bool SPIN>
__device__ __forceinline__ f2 alm_value(const MixArgs &a, int64_t ci, int v) {
  if (SPIN) {
    const float4 q = __ldg(a.alm32 + (int64_t)(2 * (v / 4) + ((v & 2) ? 1 : 0)) * a.ncoef + ci);
    return (v & 1) ? f2{q.z, q.w} : f2{q.x, q.y};
  }
  const float4 q = __ldg(a.alm32 + (int64_t)(v / 2) * a.ncoef + ci);
  return (v & 1) ? f2{q.z, q.w} : f2{q.x, q.y};
}

// the double-float a_lm value v from a staged degree row (coefficients, then the tables)
template <int NJ, bool SPIN>
__device__ __forceinline__ f2 staged_value(const float4 *row, int v) {
  const float4 q = SPIN ? row[2 + 2 * (v / 4) + ((v & 2) ? 1 : 0)] : row[2 + v / 2];
  return (v & 1) ? f2{q.z, q.w} : f2{q.x, q.y};
}

// Column bounds of one window (degrees lw0..lw1): umax[v] = max |value v| over
// the window (atomically, as FP32 bit patterns of non-negative numbers).  The
// caller synchronises before the bounds are read.
template <int NJ, bool SPIN>
__device__ __forceinline__ void window_bounds(const MixArgs &a, int64_t co, int lw0, int lw1, float *umax) {
  using S = Shape<NJ, SPIN>;
  const int v = threadIdx.x % S::NV;
  float mx = 0.f;
  for (int l = lw0 + (int)threadIdx.x / S::NV; l <= lw1; l += kRows / S::NV)
    mx = fmaxf(mx, fabsf(alm_value<NJ, SPIN>(a, co + l, v).h));
  // lanes holding the same v differ in the bits above log2(NV): reduce over them
#pragma unroll
  for (int o = S::NV; o < 32; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) < S::NV) atomicMax(reinterpret_cast<int *>(umax) + v, __float_as_int(mx));
}

// The a_lm digit stacks of a K-step from its staged rows (zero past lmax): value v
// of degree lb + k split into kAlmDigits digits on its window's grid and written,
// with the parity sign s = (-1)^(l - l0) where the column needs it, into the rows
// of the columns that read it (see the column layout in tc_syn_body).  Set t's
// stack holds NDT digit tiles of NCW rows, digit j at rows (j + 1) NCW ..; rows no
// value writes (the other set's columns, padding columns, the tile of digit -1)
// stay zero from the kernel's start.
template <int NJ, bool SPIN>
__device__ __forceinline__ void build_b(const float4 *stg, const float *umax, unsigned char *Bt) {
  using S = Shape<NJ, SPIN>;
  // byte offset of (row r of the stack, degree k) in the K-major core-matrix layout
  auto at = [](int r, int k) { return (r / 8) * 256 + (r % 8) * 16 + (k / 8) * 128 + (k % 8) * 2; };
  for (int t = threadIdx.x; t < kK * S::NV; t += kRows) {
    const int k = t % kK, v = t / kK;
    const f2 x = staged_value<NJ, SPIN>(stg + k * S::ROW, v);  // zero past lmax
    const float s0 = pow2_above(umax[v]) * 98304.0f;  // 1.5 * 2^23 * (bound * 2^-7)
    float d[kAlmDigits];
    float r = x.h;
    d[0] = round_to(r, s0);
    r = __fsub_rn(r, d[0]);
    d[1] = round_to(r, s0 * 0x1p-8f);
    r = __fsub_rn(r, d[1]);
    d[2] = round_to(r, s0 * 0x1p-16f);
    r = __fadd_rn(__fsub_rn(r, d[2]), x.l);
    d[3] = round_to(r, s0 * 0x1p-24f);
    r = __fsub_rn(r, d[3]);
    d[4] = round_to(r, s0 * 0x1p-32f);
    r = __fsub_rn(r, d[4]);
    d[5] = round_to(r, s0 * 0x1p-40f);
    const bool odd = k & 1;
    // (set, column) pairs of this value; spin: P.re -> (+, 8j) and (-, 8j+6) signed,
    // P.im -> (+, 8j+1) and (-, 8j+7) signed, M.re -> (+, 8j+2) signed and (-, 8j+4),
    // M.im -> (+, 8j+3) signed and (-, 8j+5); spin 0: the even- or odd-l column of its job
    int col0, col1 = 0, neg0 = 0, neg1 = 0, zcol = 0;
    if (SPIN) {
      const int j = v / 4, c = v % 4;
      col0 = 8 * j + c;
      col1 = 8 * j + (c < 2 ? 6 + c : 2 + c);
      neg0 = (c >= 2) && odd;
      neg1 = (c < 2) && odd;
    } else {
      const int j = v / 2, c = v % 2;
      col0 = 4 * j + (odd ? 2 : 0) + c;
      zcol = 4 * j + (odd ? 0 : 2) + c;
    }
#pragma unroll
    for (int dj = 0; dj < kAlmDigits; ++dj) {
      const int r = (dj + 1) * S::NCW;
      *reinterpret_cast<uint16_t *>(Bt + at(r + col0, k)) = bf16_of(neg0 ? -d[dj] : d[dj]);
      if (SPIN)
        *reinterpret_cast<uint16_t *>(Bt + S::NDT * S::DTILE + at(r + col1, k)) = bf16_of(neg1 ? -d[dj] : d[dj]);
      else
        *reinterpret_cast<uint16_t *>(Bt + at(r + zcol, k)) = 0;
    }
  }
}

}  // namespace tc

// ---------------------------------------------------------------------------
// synthesis, spin 0 and spin s
//
// Columns of the product (per job j): spin, 8j + {0,1} N1 = sum P l+, {2,3}
// S4 = sum s M l+, {4,5} N2 = sum M l-, {6,7} S3 = sum s P l- (re, im; s =
// (-1)^(l - l0), P = E + iB, M = E - iB); spin 0, 4j + {0,1} the even-l and
// 4j + {2,3} the odd-l sums of a_lm lambda.  The +s digits (A set 0) meet B rows
// holding P, s M; the -s digits (A set 1) rows holding M, s P.
// ---------------------------------------------------------------------------
template <int NJ, bool SPIN>
__device__ __forceinline__ void tc_syn_body(const TcArgs &ta, const int2 item, unsigned char *smem) {
  using S = tc::Shape<NJ, SPIN>;
  constexpr int NL = S::NL, NCOL = S::NCOL;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const MixArgs &a = ta.m;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int mi = item.x;
  const int p = item.y + tid;
  const bool valid = p < a.npairs;
  const int m = a.mval[mi];
  const int s = a.spin, as = s < 0 ? -s : s;
  const int l0 = m > as ? m : as, lmax = a.lmax;
  const int nks = (lmax - l0 + tc::kK) / tc::kK;
  const int64_t co = a.coef_off[mi] - l0;
  const float4 *__restrict__ cf = a.coef32 + 2 * co;
  unsigned char *const Abuf = smem;
  float4 *const stage = reinterpret_cast<float4 *>(smem + S::A_BYTES);
  unsigned char *const Bt = smem + S::A_BYTES + S::ST_BYTES;
  f2 *const accs = reinterpret_cast<f2 *>(Bt + S::B_BYTES);  // column c of this pair at accs[c * 128 + tid]
  float *const umax = reinterpret_cast<float *>(Bt + S::B_BYTES + S::ACC_BYTES);

  // the staged rows of K-step ks: thread t loads entries t, t + 128, ... (zero past lmax)
  float4 pf[S::PF];
  auto prefetch = [&](int ks) {
    const int lb = l0 + ks * tc::kK;
#pragma unroll
    for (int i = 0; i < S::PF; ++i) {
      const int e = tid + i * tc::kRows;
      pf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e < S::STG) {
        const int k = e / S::ROW, c = e % S::ROW, l = lb + k;
        if (l <= lmax) pf[i] = c < 2 ? __ldg(cf + 2 * l + c) : __ldg(a.alm32 + (int64_t)(c - 2) * a.ncoef + co + l);
      }
    }
  };
  auto stage_store = [&](int ks) {
    float4 *dst = stage + (ks & 1) * S::STG;
#pragma unroll
    for (int i = 0; i < S::PF; ++i) {
      const int e = tid + i * tc::kRows;
      if (e < S::STG) dst[e] = pf[i];
    }
  };
  __shared__ int kstart[tc::kRows / 32];
  // the K-step (block of 16 degrees) at which this pair's terms start (join record);
  // the CTA starts at its pairs' earliest
  const float4 *jrec = a.join + ((size_t)mi * a.npairs + (valid ? p : 0)) * 3;
  const int lj = valid ? __float_as_int(__ldg(jrec + 2).z) : lmax + 1;
  {
    const int kj = lj <= lmax ? (lj - l0) / tc::kK : nks;
    const int wmin = __reduce_min_sync(0xffffffffu, kj);
    if ((tid & 31) == 0) kstart[warp] = wmin;
  }
  if (warp == 0) tc::tmem_alloc(&tslot, S::TCOLS);
  if (tid == 0) tc::bar_init(&mbar);
  for (int i = tid; i < S::B_BYTES / 16; i += tc::kRows) reinterpret_cast<uint4 *>(Bt)[i] = make_uint4(0, 0, 0, 0);
  if (tid < 2 * S::NV) umax[tid] = 0.f;
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = tslot;
  const uint32_t lane = tbase + ((uint32_t)(warp * 32) << 16);
  int ks0 = kstart[0];
#pragma unroll
  for (int w = 1; w < tc::kRows / 32; ++w) ks0 = min(ks0, kstart[w]);
  if (ks0 < nks) {  // its rows; the first K-step's window barrier orders them before any read
    prefetch(ks0);
    stage_store(ks0);
  }
#pragma unroll
  for (int c = 0; c < NCOL; ++c) accs[c * tc::kRows + tid] = f2{0.f, 0.f};

  // recursion state (as in the double-float synthesis): +s values lpc/lpp, -s lmc/lmp,
  // zero until the pair joins (no terms, and a recursion of zeros)
  const PairDev pd = a.pairs[valid ? p : 0];
  const f3 x = f3_of(pd.x);
  f2 lpc = {0.f, 0.f}, lmc = {0.f, 0.f}, lpp = {0.f, 0.f}, lmp = {0.f, 0.f};
  int scp = 0, scm = 0;
  // digit grid of Lambda: magic constants of the quanta u 2^-7, u 2^-15, u 2^-23,
  // u the pair's own bound from its join record (the plan-wide bound until it joins)
  float ls0 = ta.lam_bound * 98304.0f, ls1 = ls0 * 0x1p-8f, ls2 = ls0 * 0x1p-16f;
  float racc[NCOL];
#pragma unroll
  for (int c = 0; c < NCOL; ++c) racc[c] = 0.f;

  // accumulation weight of the +s / -s values (see weight() in mixed_common.cuh): 1 at
  // scale 0, 2^-104 at scale -1, 0 below; scales change only at the rescale checks
  auto wfac = [](int sc) { return sc == 0 ? 1.f : (sc == -1 ? kScaleFactor32 : 0.f); };
  float wfp = wfac(scp), wfm = wfac(scm);
  bool settled = false;  // every lane of the warp at scale 0 (warp-uniform; scales only rise)

  // kPack degrees from rows (lb - l0 even): digits packed per pair of degrees into
  // pk[set][digit][q / 2], remainders contracted into racc, recursion advanced.
  // Every second degree the warp votes: if every lane's values are negligible for
  // the next two steps (as in the double-float kernels) the digits are zero and
  // only the recursion runs.
  auto part = [&](const float4 *rows, uint32_t (&pk)[NL][tc::kLamDigits][tc::kPack / 2]) {
    float dlo[NL][tc::kLamDigits];
    bool dead = false;
#pragma unroll
    for (int q = 0; q < tc::kPack; ++q) {
      // past lmax the staged rows are zero: the recursion runs on zero coefficients
      // (its values become zero one degree later) and meets zero a_lm, so those
      // degrees add nothing and need no test
      const bool odd = q & 1;
      if (!odd) dead = !settled && __all_sync(0xffffffffu, negligible(lpc, scp) && (!SPIN || negligible(lmc, scm)));
      const float4 *row = rows + q * S::ROW;  // this degree's staged coefficients and a_lm
      if (!dead) {
        f2 w[NL];
        w[0] = f2{lpc.h * wfp, lpc.l * wfp};
        if (SPIN) w[1] = f2{lmc.h * wfm, lmc.l * wfm};
        float rr[NL];
#pragma unroll
        for (int t = 0; t < NL; ++t) {
          const float d0 = tc::round_to(w[t].h, ls0);
          float r = __fsub_rn(w[t].h, d0);
          const float d1 = tc::round_to(r, ls1);
          r = __fsub_rn(r, d1);
          const float d2 = tc::round_to(r, ls2);
          rr[t] = __fadd_rn(__fsub_rn(r, d2), w[t].l);
          if (!odd) {
            dlo[t][0] = d0;
            dlo[t][1] = d1;
            dlo[t][2] = d2;
          } else {
            pk[t][0][q / 2] = tc::pack_bf16(dlo[t][0], d0);
            pk[t][1][q / 2] = tc::pack_bf16(dlo[t][1], d1);
            pk[t][2][q / 2] = tc::pack_bf16(dlo[t][2], d2);
          }
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          if (SPIN) {
            const float4 P = row[2 + 2 * j];
            const float4 M = row[3 + 2 * j];
            const float rp = rr[0], rm = rr[1], sp = odd ? -rr[0] : rr[0], sm = odd ? -rr[1] : rr[1];
            racc[8 * j + 0] = __fmaf_rn(rp, P.x, racc[8 * j + 0]);
            racc[8 * j + 1] = __fmaf_rn(rp, P.z, racc[8 * j + 1]);
            racc[8 * j + 2] = __fmaf_rn(sp, M.x, racc[8 * j + 2]);
            racc[8 * j + 3] = __fmaf_rn(sp, M.z, racc[8 * j + 3]);
            racc[8 * j + 4] = __fmaf_rn(rm, M.x, racc[8 * j + 4]);
            racc[8 * j + 5] = __fmaf_rn(rm, M.z, racc[8 * j + 5]);
            racc[8 * j + 6] = __fmaf_rn(sm, P.x, racc[8 * j + 6]);
            racc[8 * j + 7] = __fmaf_rn(sm, P.z, racc[8 * j + 7]);
          } else {
            const float4 v = row[2 + j];
            const int c = 4 * j + (odd ? 2 : 0);
            racc[c] = __fmaf_rn(rr[0], v.x, racc[c]);
            racc[c + 1] = __fmaf_rn(rr[0], v.z, racc[c + 1]);
          }
        }
      } else {  // zero digits (negligible values)
#pragma unroll
        for (int t = 0; t < NL; ++t) {
          if (!odd) {
            dlo[t][0] = dlo[t][1] = dlo[t][2] = 0.f;
          } else {
            pk[t][0][q / 2] = tc::pack_bf16(dlo[t][0], 0.f);
            pk[t][1][q / 2] = tc::pack_bf16(dlo[t][1], 0.f);
            pk[t][2][q / 2] = tc::pack_bf16(dlo[t][2], 0.f);
          }
        }
      }
      {
        const float4 u = row[0], v = row[1];
        const Coef32 cc = {{u.x, u.y}, {u.z, u.w}, {v.x, v.y}};
        const f2 t = mul(cc.a, x);
        const f2 nc = neg(cc.c);
        if (SPIN) {
          const f2 np_ = dot3(t, lpc, cc.ak, lpc, nc, lpp);
          const f2 nm_ = dot3(t, lmc, neg(cc.ak), lmc, nc, lmp);
          lpp = lpc;
          lpc = np_;
          lmp = lmc;
          lmc = nm_;
        } else {
          const f2 ln = dot2(t, lpc, nc, lpp);
          lpp = lpc;
          lpc = ln;
        }
      }
    }
  };
  // enhanced exponent: rescale every eight degrees (see mixed_common.cuh)
  auto rescale = [&]() {
    if (settled) return;
    if (scp < 0 && fabsf(lpc.h) > kScaleUp32) {
      lpc = {lpc.h * kScaleFactor32, lpc.l * kScaleFactor32};
      lpp = {lpp.h * kScaleFactor32, lpp.l * kScaleFactor32};
      ++scp;
    }
    if (SPIN && scm < 0 && fabsf(lmc.h) > kScaleUp32) {
      lmc = {lmc.h * kScaleFactor32, lmc.l * kScaleFactor32};
      lmp = {lmp.h * kScaleFactor32, lmp.l * kScaleFactor32};
      ++scm;
    }
    wfp = wfac(scp);
    wfm = wfac(scm);
    settled = __all_sync(0xffffffffu, scp == 0 && scm == 0);
  };
  // this thread's digits of degrees q0 .. q0 + kPack - 1 of the K-step into the A tiles
  auto store_a = [&](int q0, const uint32_t (&pk)[NL][tc::kLamDigits][tc::kPack / 2]) {
#pragma unroll
    for (int t = 0; t < NL; ++t)
#pragma unroll
      for (int i = 0; i < tc::kLamDigits; ++i) {
        unsigned char *dst = Abuf + (t * tc::kLamDigits + i) * tc::kATile + (tid / 8) * 256 + (q0 / 8) * 128 +
                             (tid % 8) * 16 + (q0 % 8) * 2;
        if (tc::kPack == 8)
          *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(pk[t][i]);
        else
          *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(pk[t][i]);
      }
  };

  // the MMAs of one K-step, issued in order by one thread: for each Lambda set t and
  // digit i, the a_lm digit windows (j0, j0 + 1), j0 = -(i mod 2), j0 + 2, ... up to
  // the last digit with i + j <= 5, into levels (i + j0, i + j0 + 1); in a window's
  // first K-step the set-0, digit-0 products come first and overwrite levels 0 .. 5
  // (every level written), the rest accumulate.  The zero tile of digit -1 fills
  // the odd windows' first halves; the i = 2 windows end at digit 3.
  const uint64_t adesc0 = tc::mat_desc(tc::smem_u32(Abuf), 128, 256);
  const uint64_t bdesc0 = tc::mat_desc(tc::smem_u32(Bt), 128, 256);
  auto issue = [&](int ks) {
    tc::fence_after();
    constexpr uint32_t idesc = tc::instr_desc(tc::kRows, S::N);
    const bool first = (ks % tc::kWin) == 0 || ks == ks0;
#pragma unroll
    for (int t = 0; t < NL; ++t)
#pragma unroll
      for (int i = 0; i < tc::kLamDigits; ++i)
#pragma unroll
        for (int j0 = -(i & 1); j0 <= tc::kAlmDigits - 1 && i + j0 < tc::kLevels; j0 += 2) {
          const uint64_t ad = adesc0 + (uint64_t)(((t * tc::kLamDigits + i) * tc::kATile) >> 4);
          const uint64_t bd = bdesc0 + (uint64_t)((t * S::NDT * S::DTILE + (j0 + 1) * S::DTILE) >> 4);
          tc::mma_bf16(tbase + (i + j0) * S::NCW, ad, bd, idesc, (first && t == 0 && i == 0) ? 0u : 1u);
        }
    tc::mma_commit(&mbar);
  };

  // after a window: the six levels of this thread's lane plus the remainder sums,
  // added to the double-float column sums
  auto readout = [&]() {
#pragma unroll
    for (int c0 = 0; c0 < NCOL; c0 += 8) {
      uint32_t dv[tc::kLevels][8];
#pragma unroll
      for (int k = 0; k < tc::kLevels; ++k) tc::tmem_ld8(lane + k * S::NCW + c0, dv[k]);
      tc::tmem_wait_ld();
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (c0 + c >= NCOL) break;
        f2 t = {__uint_as_float(dv[0][c]), 0.f};
#pragma unroll
        for (int k = 1; k < tc::kLevels; ++k) t = f2_add_lazy(t, f2{__uint_as_float(dv[k][c]), 0.f});
        t = f2_add_lazy(t, f2{racc[c0 + c], 0.f});
        racc[c0 + c] = 0.f;
        f2 &acc = accs[(c0 + c) * tc::kRows + tid];
        acc = f2_add(acc, t);
      }
    }
  };

  int ncommit = 0, nwaited = 0;
  bool ok = true;
  for (int ks = ks0; ks < nks; ++ks) {
    const int lb = l0 + ks * tc::kK;
    if (ks % tc::kWin == 0 || ks == ks0) {  // column bounds of this window's a_lm (from lb on)
      float *um = umax + ((ks / tc::kWin) & 1) * S::NV;
      if (tid < S::NV) umax[(((ks / tc::kWin) & 1) ^ 1) * S::NV + tid] = 0.f;  // the other window's, for later
      const int lw1 = l0 + (ks / tc::kWin + 1) * tc::kWin * tc::kK - 1;
      tc::window_bounds<NJ, SPIN>(a, co, lb, lw1 < lmax ? lw1 : lmax, um);
      __syncthreads();
    }
    if (lj == lb) {  // this pair joins: the recursion state where its terms start
      const JoinRec r = ld_join(jrec);
      lpc = r.lpc;
      lpp = r.lpp;
      lmc = r.lmc;
      lmp = r.lmp;
      scp = r.scp;
      scm = r.scm;
      wfp = wfac(scp);
      wfm = wfac(scm);
      ls0 = __int_as_float((127 + r.lexp) << 23) * 98304.0f;
      ls1 = ls0 * 0x1p-8f;
      ls2 = ls0 * 0x1p-16f;
    }
    if (__any_sync(0xffffffffu, lj == lb)) settled = __all_sync(0xffffffffu, scp == 0 && scm == 0);
    // a warp none of whose lanes has joined holds zeros: it skips the recursion
    const bool wlive = __any_sync(0xffffffffu, lj <= lb);
    const float4 *rows = stage + (ks & 1) * S::STG;
    if (ks + 1 < nks) prefetch(ks + 1);  // its latency hides behind this K-step's work
    bool fail = false;
#pragma unroll 1
    for (int q0 = 0; q0 < tc::kK; q0 += tc::kPack) {
      uint32_t pk[NL][tc::kLamDigits][tc::kPack / 2];
      if (wlive) {
        part(rows + q0 * S::ROW, pk);
      } else {  // no lane of the warp has joined: zero digits, and nothing to advance
#pragma unroll
        for (int t = 0; t < NL; ++t)
#pragma unroll
          for (int i = 0; i < tc::kLamDigits; ++i)
#pragma unroll
            for (int q = 0; q < tc::kPack / 2; ++q) pk[t][i][q] = 0u;
      }
      if (q0 % 8 == tc::kPack % 8) rescale();  // after every eight degrees
      // the previous K-step's MMAs read the A and B tiles: wait for them before
      // the first write (they have long finished by now)
      if (q0 == 0 && ncommit > nwaited) {
        fail = !tc::bar_wait(&mbar, (uint32_t)(ncommit - 1) & 1u);
        nwaited = ncommit;
      }
      if (!fail) store_a(q0, pk);
    }
    if (!fail) tc::build_b<NJ, SPIN>(rows, umax + ((ks / tc::kWin) & 1) * S::NV, Bt);
    if (ks + 1 < nks) stage_store(ks + 1);  // its buffer's last readers finished before the previous barrier
    tc::fence_async_smem();
    if (__syncthreads_or(fail)) {
      ok = false;
      break;
    }
    if (tid == tc::kIssuerThread) issue(ks);
    ++ncommit;
    if (ks % tc::kWin == tc::kWin - 1 || ks == nks - 1) {
      fail = !tc::bar_wait(&mbar, (uint32_t)(ncommit - 1) & 1u);
      nwaited = ncommit;
      if (__syncthreads_or(fail)) {
        ok = false;
        break;
      }
      tc::fence_after();
      readout();
      tc::fence_before();
    }
  }
  if (!ok) {  // a wait gave up: flag it, give the MMAs in flight a bounded wait, release TMEM
    if (tid == 0) atomicOr(ta.err, 1);
    if (ncommit > nwaited) tc::bar_wait(&mbar, (uint32_t)(ncommit - 1) & 1u);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tbase, S::TCOLS);
  if (!ok || !valid) return;
  auto colsum = [&](int c) { return f2_val(accs[c * tc::kRows + tid]); };

  if (SPIN) {
    const double sig = (as & 1) ? -1.0 : 1.0;
    const double h0 = ((l0 + m) & 1) ? -0.5 : 0.5;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const double n1r = colsum(8 * j + 0), n1i = colsum(8 * j + 1);
      const double s4r = colsum(8 * j + 2), s4i = colsum(8 * j + 3);
      const double n2r = colsum(8 * j + 4), n2i = colsum(8 * j + 5);
      const double s3r = colsum(8 * j + 6), s3i = colsum(8 * j + 7);
      const double ar = n1r + sig * n2r, ai = n1i + sig * n2i;
      const double br = sig * n2r - n1r, bi = sig * n2i - n1i;
      const double cr = s3r + sig * s4r, ci = s3i + sig * s4i;
      const double dr = sig * s4r - s3r, di = sig * s4i - s3i;
      double2 qn = make_double2(-0.5 * ar, -0.5 * ai);
      double2 un = make_double2(0.5 * bi, -0.5 * br);
      double2 qs = make_double2(-h0 * cr, -h0 * ci);
      double2 us = make_double2(h0 * di, -h0 * dr);
      if (m == 0) qn.y = qs.y = un.y = us.y = 0.0;
      double2 *oq = a.phase + (((size_t)(2 * j) * a.nm + mi) * a.npairs + p) * 2;
      double2 *ou = a.phase + (((size_t)(2 * j + 1) * a.nm + mi) * a.npairs + p) * 2;
      oq[0] = qn;
      oq[1] = qs;
      ou[0] = un;
      ou[1] = us;
    }
  } else {
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const double e0 = colsum(4 * j + 0), e1 = colsum(4 * j + 1);
      const double o0 = colsum(4 * j + 2), o1 = colsum(4 * j + 3);
      double2 fn = make_double2(e0 + o0, e1 + o1), fs = make_double2(e0 - o0, e1 - o1);
      if (m == 0) fn.y = fs.y = 0.0;
      double2 *o = a.phase + (((size_t)j * a.nm + mi) * a.npairs + p) * 2;
      o[0] = fn;
      o[1] = fs;
    }
  }
}

}  // namespace sht

namespace sht {

template <int NJ, bool SPIN>
__global__ void __launch_bounds__(tc::kRows, tc::Shape<NJ, SPIN>::MINB) tc_syn(TcArgs ta) {
  extern __shared__ __align__(128) unsigned char tc_smem[];
  tc_syn_body<NJ, SPIN>(ta, ta.m.syn_items[blockIdx.x], tc_smem);
}

// batches: item (mi, first pair, -, record); the record holds the plan's arguments
template <int NJ, bool SPIN>
__global__ void __launch_bounds__(tc::kRows, tc::Shape<NJ, SPIN>::MINB)
    tc_syn_batch(const TcArgs *__restrict__ args, const int4 *__restrict__ items) {
  extern __shared__ __align__(128) unsigned char tc_smem[];
  const int4 it = items[blockIdx.x];
  tc_syn_body<NJ, SPIN>(args[it.w], make_int2(it.x, it.y), tc_smem);
}

template <int NJ, bool SPIN>
static cudaError_t tc_set_smem() {
  // the request, and a shared-memory carveout that lets the compiled number of CTAs fit
  cudaError_t e = cudaFuncSetAttribute(tc_syn_batch<NJ, SPIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       tc::Shape<NJ, SPIN>::SMEM_LAUNCH);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_syn<NJ, SPIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc::Shape<NJ, SPIN>::SMEM_LAUNCH);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_syn_batch<NJ, SPIN>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_syn<NJ, SPIN>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  return e;
}

// shared-memory attributes of every instance (once per device, at plan time)
cudaError_t tc_prepare_device() {
  cudaError_t e = tc_set_smem<1, false>();
  if (e == cudaSuccess) e = tc_set_smem<2, false>();
  if (e == cudaSuccess) e = tc_set_smem<4, false>();
  if (e == cudaSuccess) e = tc_set_smem<8, false>();
  if (e == cudaSuccess) e = tc_set_smem<1, true>();
  if (e == cudaSuccess) e = tc_set_smem<2, true>();
  if (e == cudaSuccess) e = tc_set_smem<4, true>();
  return e;
}

bool tc_supported(int spin, int njobs_pad) {
  return spin == 0 ? njobs_pad <= 8 : njobs_pad <= 4;
}

float tc_lambda_bound(int lmax) {
  // |sLambda_lm| <= sqrt((2l + 1) / (4 pi)) (|d^l| <= 1) up to l = lmax + 1 (the
  // kernel computes one value past lmax); the next power of two above it, with
  // room for the recursion's rounding
  const double b = sqrt((2.0 * lmax + 3.0) / (4.0 * M_PI)) * (1.0 + 1e-6);
  return (float)exp2(ceil(log2(b)));
}

size_t tc_args_size() { return sizeof(TcArgs); }

void leg_tc_fill_args(const sht_plan_s *P, int polar, int ptr_off, void *out) {
  TcArgs ta;
  leg_mixed_fill_args(P, polar, ptr_off, &ta.m);
  ta.lam_bound = P->tc_lam_bound;
  ta.err = P->d_err;
  memcpy(out, &ta, sizeof(ta));
}

cudaError_t launch_leg_tc_batch(int spin, int nj, const void *targs, const int4 *items, int n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const TcArgs *a = static_cast<const TcArgs *>(targs);
  if (spin == 0) {
    switch (nj) {
      case 1: tc_syn_batch<1, false><<<n, tc::kRows, tc::Shape<1, false>::SMEM_LAUNCH, st>>>(a, items); break;
      case 2: tc_syn_batch<2, false><<<n, tc::kRows, tc::Shape<2, false>::SMEM_LAUNCH, st>>>(a, items); break;
      case 4: tc_syn_batch<4, false><<<n, tc::kRows, tc::Shape<4, false>::SMEM_LAUNCH, st>>>(a, items); break;
      case 8: tc_syn_batch<8, false><<<n, tc::kRows, tc::Shape<8, false>::SMEM_LAUNCH, st>>>(a, items); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (nj) {
      case 1: tc_syn_batch<1, true><<<n, tc::kRows, tc::Shape<1, true>::SMEM_LAUNCH, st>>>(a, items); break;
      case 2: tc_syn_batch<2, true><<<n, tc::kRows, tc::Shape<2, true>::SMEM_LAUNCH, st>>>(a, items); break;
      case 4: tc_syn_batch<4, true><<<n, tc::kRows, tc::Shape<4, true>::SMEM_LAUNCH, st>>>(a, items); break;
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_leg_tc_syn(const sht_plan_s *P, const void *mixargs, int n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  TcArgs ta;
  memcpy(&ta.m, mixargs, sizeof(MixArgs));
  ta.lam_bound = P->tc_lam_bound;
  ta.err = P->d_err;
  const int nj = P->njobs_pad;
  if (P->spin == 0) {
    switch (nj) {
      case 1: tc_syn<1, false><<<n, tc::kRows, tc::Shape<1, false>::SMEM_LAUNCH, st>>>(ta); break;
      case 2: tc_syn<2, false><<<n, tc::kRows, tc::Shape<2, false>::SMEM_LAUNCH, st>>>(ta); break;
      case 4: tc_syn<4, false><<<n, tc::kRows, tc::Shape<4, false>::SMEM_LAUNCH, st>>>(ta); break;
      case 8: tc_syn<8, false><<<n, tc::kRows, tc::Shape<8, false>::SMEM_LAUNCH, st>>>(ta); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (nj) {
      case 1: tc_syn<1, true><<<n, tc::kRows, tc::Shape<1, true>::SMEM_LAUNCH, st>>>(ta); break;
      case 2: tc_syn<2, true><<<n, tc::kRows, tc::Shape<2, true>::SMEM_LAUNCH, st>>>(ta); break;
      case 4: tc_syn<4, true><<<n, tc::kRows, tc::Shape<4, true>::SMEM_LAUNCH, st>>>(ta); break;
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

}  // namespace sht
