// legendre_tc_ana.cu -- the mixed form's Legendre analysis (Eq. ana1) with the
// contraction over ring pairs on the tensor cores (tcgen05).
//
// For one m and a tile of 128 ring pairs the analysis adds, for every degree l,
// a[l][c] = sum_p G[c][p] Lambda[p][l]: the columns c are the phase values of the
// ring pairs combined for the parity of l - l0 and the spin (Sect. 3.2's loop over
// rings inside the loop over l, Fig. 2), Lambda comes from the double-float
// recursion of Sect. 4.1, one thread per ring pair walking l.  The contraction
// runs transposed, D[c][l] = sum_p G[c][p] Lambda[p][l]: M = the columns' digit
// rows, K = the ring pairs, N = degrees, so that each thread writes its own pair's
// values along N (the Lambda operand in the MN-major layout) and the G operand is
// built once per tile.  Both operands are split exactly into bf16 digits on common
// grids (an Ozaki-style error-free split):
//
//  * Lambda / u_p = L0 + ... + L5 on the grid 2^(-7-8i), u_p a power of two
//    bounding the pair's true values from its join block on (join record), so
//    |Lambda / u_p| < 1; the pair's factor u_p moves into its G values.
//  * G'[c][p] = G[c][p] u_p = G0 + ... + G5 on the grid v_c 2^(-7-8j), v_c the
//    power of two above column c's largest |G'| over the tile.
//  * Every product Gj Li is a multiple of v_c 2^(-14-8(i+j)); a digit is at most
//    128 of its quanta (192 for digit 3, which takes the low word), so a sum over
//    the tile's K = 128 or 256 pair entries stays below 256 * 192^2 < 2^24 quanta
//    and the FP32 accumulation is exact whatever its order.
//
// One MMA per 16 pair entries: M = 64 rows (column c's six G digits and two zero
// rows at rows 8c .. 8c + 7), N = 48 (the six Lambda digits of 8 degrees), so D
// holds every digit product G_j L_i of a column and degree, each an exact sum; the
// products with i + j <= 2 are added in double-float, those with 3 <= i + j <= 6 in
// FP32 (below 2^-24 of the sum), the rest dropped (below 2^-56).  Measured at spin
// 2, lmax 4095 on GB300 (double-float analysis 76.5 ms): three MMAs of N = 16 per 16
// entries whose A row shifts summed the levels on the tensor cores, 92 ms (each
// read 4 KB of A from shared memory); one MMA of N = 48 at M = 128, 86 ms; M = 64
// and waits that suspend the waiting warp, 80 ms; no per-degree negligibility vote
// (the join records cover it), 73.8 ms.
//
// Each warp owns the K entries of its 32 pairs: it writes their Lambda digits and
// issues their MMAs itself (lane 0), with no CTA barrier per block.  Two TMEM
// accumulators of 48 columns alternate between blocks of 8 degrees; mbarriers
// order the steps: a warp's own commits free its Lambda tiles, every warp's
// commit (or plain arrival for a warp with no joined pair) fills an accumulator,
// and the warps holding its rows (M = 64 puts D row r in TMEM lane 32 (r / 16) +
// r % 16: warp w holds columns 2w and 2w + 1) release it after reading and zeroing
// it.  Every
// wait is bounded; a wait that gives up flags the plan's status word and stops the
// CTA.
#include "tcgen05.cuh"

namespace sht {
namespace tca {

constexpr int kPairs = 128;      // ring pairs per CTA = threads
constexpr int kWarps = kPairs / 32;
constexpr int kBlk = 8;          // degrees per block
constexpr int kDig = 6;          // digits of Lambda / u_p and of G'
constexpr int kN = kDig * kBlk;  // MMA N: every Lambda digit of the block's degrees
constexpr int kColRows = 8;      // A rows per column: its six G digits, two zero rows
constexpr int kDCols = 64;       // TMEM columns per accumulator (kN used)
constexpr int kM = 64;           // MMA M: the columns' digit rows
constexpr int kEStride = kN + 4; // floats per staged D row (rows 16 bytes off the banks of the next)
constexpr int kKStride = 144;    // bytes between 8-pair K-groups of the Lambda tiles (stores without bank conflicts)

// Columns per job j: 4j + {0, 1} and 4j + {2, 3} (re, im of the two sums the
// kernel below describes); K entries 0..127 hold the pairs' +s (or spin-0) values,
// 128..255 the -s values times (-1)^(l - l0).  Column c's six G digit rows and
// two zero rows make 8 rows of A and of D.
template <int NJ, bool SPIN>
struct AnaShape {
  static constexpr int NSET = SPIN ? 2 : 1;
  static constexpr int NC = 4 * NJ;
  static constexpr int KG = NSET * kPairs / 8;  // 8-entry K-groups
  // MMA M = 64: D row r lands in TMEM lane 32 (r / 16) + r % 16 (measured).
  // Column c's rows are A and D rows 8c .. 8c + 7, so warp w holds columns 2w and
  // 2w + 1 in lanes 0 .. 15; the rows of one K-group are contiguous (SBO = 128,
  // LBO = the rows' bytes).
  static constexpr int NREAD = NC / 2;        // warps holding D rows
  static constexpr int A_LBO = NC * kColRows * 16;  // bytes between K-groups
  static constexpr int A_SBO = 128;                 // bytes between 8-row groups
  static constexpr int A_BYTES = KG * A_LBO;
  // byte offset of (column c, digit row j, K-group h)
  __host__ __device__ static constexpr int a_at(int c, int j, int h) { return h * A_LBO + (kColRows * c + j) * 16; }
  static constexpr int B_SBO = KG * kKStride;  // bytes between the 8-degree N-groups (one per digit)
  static constexpr int B_BYTES = kDig * B_SBO;
  static constexpr int EROWS = 2 * kColRows;  // staged D rows per reading warp: lanes 0 .. 15
  static constexpr int E_BYTES = NREAD * EROWS * kEStride * 4;
  static constexpr int SMEM = A_BYTES + B_BYTES + E_BYTES;
  // at most 512 / 128 CTAs per SM, so that their TMEM allocations never wait
  static constexpr int SMEM_FLOOR = (228 * 1024) / 5 - 1024 + 1;
  static constexpr int SMEM_LAUNCH = SMEM > SMEM_FLOOR ? SMEM : SMEM_FLOOR;
  static constexpr int V = (SPIN ? 4 : 2) * NJ;  // partial sums per degree
  static constexpr int MINB = SMEM_LAUNCH <= 57 * 1024 ? 4 : (SMEM_LAUNCH <= 75 * 1024 ? 3 : 2);
  static_assert(kColRows * NC <= kM && NREAD <= kWarps, "columns within the MMA's rows");
  // the MMA reads kM rows of two K-groups from a K-step's base: from the last
  // one's, inside A and the B tiles that follow it
  static_assert((KG - 1) * A_LBO + kM * 16 <= A_BYTES + B_BYTES, "A operand inside shared memory");
  static_assert(A_BYTES % 16 == 0 && B_SBO % 16 == 0, "descriptor alignment");
};

// six digits of x on the grid whose first quantum has the magic constant s0
// (1.5 * 2^23 * quantum; |x| < 2^22 quanta): each a multiple of its quantum with at
// most 8 significant bits (at most 128 quanta; 192 for d[3], after the low word
// enters)
__device__ __forceinline__ void split6(f2 x, float s0, float (&d)[kDig]) {
  float r = x.h;
  d[0] = tc::round_to(r, s0);
  r = __fsub_rn(r, d[0]);
  d[1] = tc::round_to(r, s0 * 0x1p-8f);
  r = __fsub_rn(r, d[1]);
  d[2] = tc::round_to(r, s0 * 0x1p-16f);
  r = __fadd_rn(__fsub_rn(r, d[2]), x.l);
  d[3] = tc::round_to(r, s0 * 0x1p-24f);
  r = __fsub_rn(r, d[3]);
  d[4] = tc::round_to(r, s0 * 0x1p-32f);
  r = __fsub_rn(r, d[4]);
  d[5] = tc::round_to(r, s0 * 0x1p-40f);
}

}  // namespace tca

// ---------------------------------------------------------------------------
// Columns' K entries per ring pair (mixed analysis naming: W+_N, W-_N the north
// ring's spin combinations, W+_S', W-_S' the south ring's times (-1)^(l0 + m)):
// spin, T1 = sum l+ W+_N + s l- W+_S' and s T2 = sum l+ W-_S' + s l- W-_N with
// s = (-1)^(l - l0), so the K entries are the +s values and the -s values times s,
// and T2 is s times its row; spin 0, the even-l sum over G_N + G_S and the odd-l
// sum over G_N - G_S.
// ---------------------------------------------------------------------------
template <int NJ, bool SPIN>
__device__ __forceinline__ void tc_ana_body(const TcArgs &ta, const int4 item, unsigned char *tca_smem) {
  using S = tca::AnaShape<NJ, SPIN>;
  constexpr int NSET = S::NSET, NC = S::NC, V = S::V, kDig = tca::kDig;
  __shared__ __align__(8) uint64_t full[2], freeb[2], mine[tca::kWarps];
  __shared__ uint32_t tslot;
  __shared__ unsigned vmax[NC];
  __shared__ int tstart[tca::kWarps];
  __shared__ volatile int stop;
  const MixArgs &a = ta.m;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mi = item.x, ng = item.z & 255;
  const int m = a.mval[mi];
  const int s = a.spin, as = s < 0 ? -s : s;
  const int l0 = m > as ? m : as, lmax = a.lmax, nl = lmax - l0 + 1;
  const float4 *__restrict__ cf = a.coef32 + 2 * (a.coef_off[mi] - l0);
  double *const outp = a.part + a.part_off[mi] + (int64_t)(item.z >> 8) * nl * V;
  const double sg0 = ((l0 + m) & 1) ? -1.0 : 1.0;
  unsigned char *const Abuf = tca_smem;
  unsigned char *const Bbuf = tca_smem + S::A_BYTES;
  // a reading warp's staged D rows (kN columns each; the other warps never use theirs)
  float *const Ebuf =
      reinterpret_cast<float *>(tca_smem + S::A_BYTES + S::B_BYTES) + (warp % S::NREAD) * S::EROWS * tca::kEStride;

  if (warp == 0) tc::tmem_alloc(&tslot, 2 * tca::kDCols);
  if (tid == 0) {
    tc::bar_init(&full[0], tca::kWarps);
    tc::bar_init(&full[1], tca::kWarps);
    tc::bar_init(&freeb[0], S::NREAD);  // the warps holding D rows read and release it
    tc::bar_init(&freeb[1], S::NREAD);
#pragma unroll
    for (int w = 0; w < tca::kWarps; ++w) tc::bar_init(&mine[w], 1);
    stop = 0;
  }
  // A starts at zero: rows 6 and 7 of each column (below its six digits) stay so
  for (int i = tid; i < S::A_BYTES / 16; i += tca::kPairs) reinterpret_cast<uint4 *>(Abuf)[i] = make_uint4(0, 0, 0, 0);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = tslot;
  const uint32_t tlane = tbase + ((uint32_t)(warp * 32) << 16);
  // both accumulators start at zero (ordered before any MMA by the tile's barriers)
  if (warp < S::NREAD) {
#pragma unroll
    for (int q = 0; q < 2 * tca::kN / 16; ++q) tc::tmem_zero16(tlane + (q / 3) * tca::kDCols + (q % 3) * 16);
    tc::tmem_wait_st();
  }
  tc::fence_before();

  const uint64_t adesc0 = tc::mat_desc(tc::smem_u32(Abuf), S::A_LBO, S::A_SBO);
  const uint64_t bdesc0 = tc::mat_desc(tc::smem_u32(Bbuf), tca::kKStride, S::B_SBO);
  constexpr uint32_t idesc = tc::instr_desc(tca::kM, tca::kN, true);

  int ib = 0;                    // blocks walked by the CTA over all its tiles: accumulator ib & 1
  int nmine = 0, nmine_done = 0;  // this warp's commits to mine[warp], and those waited for
  bool ok = true;
  // a bounded wait of the whole warp (false for every lane if any lane gave up)
  auto wait_warp = [&](uint64_t *bar, uint32_t parity) {
    const bool r = tc::bar_wait_or(bar, parity, &stop);
    return __all_sync(0xffffffffu, r);
  };
  auto give_up = [&]() {
    if (lane == 0) stop = 1;
    ok = false;
  };
  auto wfac = [](int sc) { return sc == 0 ? 1.f : (sc == -1 ? kScaleFactor32 : 0.f); };

#pragma unroll 1
  for (int gi = 0; gi < ng; ++gi) {
    const int tile = item.y + gi;
    const int p = tile * tca::kPairs + tid;
    const bool valid = p < a.npairs;
    const float4 *jrec = a.join + ((size_t)mi * a.npairs + (valid ? p : 0)) * 3;
    int lj = lmax + 1, lexp = 0;
    if (valid) {
      const float4 c = __ldg(jrec + 2);
      lj = __float_as_int(c.z);
      lexp = __float_as_int(c.w);
    }
    // this pair's K entries of every column, times its Lambda bound u_p = 2^lexp
    // (zero for a pair that never joins)
    double gv[NSET][NC];
#pragma unroll
    for (int t = 0; t < NSET; ++t)
#pragma unroll
      for (int c = 0; c < NC; ++c) gv[t][c] = 0.0;
    if (valid && lj <= lmax) {
      const double u = ldexp(1.0, lexp);
      const bool south = a.pairs[p].south;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        if (!SPIN) {
          const double2 *gp = a.phase + (((size_t)j * a.nm + mi) * a.npairs + p) * 2;
          const double2 gn = gp[0], gs = south ? gp[1] : make_double2(0.0, 0.0);
          gv[0][4 * j + 0] = u * (gn.x + gs.x);
          gv[0][4 * j + 1] = u * (gn.y + gs.y);
          gv[0][4 * j + 2] = u * (gn.x - gs.x);
          gv[0][4 * j + 3] = u * (gn.y - gs.y);
        } else {
          const double2 *gq = a.phase + (((size_t)(2 * j) * a.nm + mi) * a.npairs + p) * 2;
          const double2 *gu = a.phase + (((size_t)(2 * j + 1) * a.nm + mi) * a.npairs + p) * 2;
          const double2 qn = gq[0], un = gu[0];
          const double2 qs = south ? gq[1] : make_double2(0.0, 0.0), us = south ? gu[1] : make_double2(0.0, 0.0);
          // W+_N, W-_N, W+_S', W-_S' (re, im)
          const double wpn_r = qn.x - un.y, wpn_i = qn.y + un.x;
          const double wmn_r = qn.x + un.y, wmn_i = qn.y - un.x;
          const double wps_r = sg0 * (qs.x - us.y), wps_i = sg0 * (qs.y + us.x);
          const double wms_r = sg0 * (qs.x + us.y), wms_i = sg0 * (qs.y - us.x);
          gv[0][4 * j + 0] = u * wpn_r;  // T1: l+ W+_N
          gv[0][4 * j + 1] = u * wpn_i;
          gv[0][4 * j + 2] = u * wms_r;  // s T2: l+ W-_S'
          gv[0][4 * j + 3] = u * wms_i;
          gv[1][4 * j + 0] = u * wps_r;  // T1: s l- W+_S'
          gv[1][4 * j + 1] = u * wps_i;
          gv[1][4 * j + 2] = u * wmn_r;  // s T2: s l- W-_N
          gv[1][4 * j + 3] = u * wmn_i;
        }
      }
    }
    __syncthreads();  // the previous tile's products are complete (its last accumulator was read)
    if (stop) {       // read after a barrier: the same for every warp
      ok = false;
      break;
    }
    if (tid < NC) vmax[tid] = 0u;
    {
      const int wmin = __reduce_min_sync(0xffffffffu, lj);
      if (lane == 0) tstart[warp] = wmin;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NC; ++c) {  // column bounds over the tile (FP32 bit patterns of |G'|)
      float mx = 0.f;
#pragma unroll
      for (int t = 0; t < NSET; ++t) mx = fmaxf(mx, fabsf(__double2float_ru(fabs(gv[t][c]))));
      const unsigned w = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
      if (lane == 0) atomicMax(&vmax[c], w);
    }
    __syncthreads();
    int lstart = tstart[0];
#pragma unroll
    for (int w = 1; w < tca::kWarps; ++w) lstart = min(lstart, tstart[w]);
    // the G' digits of this pair into A: column c's digit j at its row j of the
    // pair's K-group, entry tid % 8 (rows 6 and 7 stay zero)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const float s0 = tc::pow2_above(__uint_as_float(vmax[c])) * 98304.0f;  // 1.5 * 2^23 * (v_c 2^-7)
#pragma unroll
      for (int t = 0; t < NSET; ++t) {
        float d[kDig];
        tca::split6(f2_of(gv[t][c]), s0, d);
        unsigned char *dst = Abuf + S::a_at(c, 0, t * (tca::kPairs / 8) + tid / 8) + (tid % 8) * 2;
#pragma unroll
        for (int j = 0; j < kDig; ++j) *reinterpret_cast<uint16_t *>(dst + j * 16) = tc::bf16_of(d[j]);
      }
    }
    if (gi == 0)  // the slot's degrees before the tile's first block (later tiles add to them)
      for (int i = tid; i < (min(lstart, lmax + 1) - l0) * V; i += tca::kPairs) outp[i] = 0.0;
    tc::fence_async_smem();
    __syncthreads();
    if (lstart > lmax) continue;

    // the walk over the tile's blocks of 8 degrees (from its pairs' earliest join)
    const f3 x = f3_of(valid ? a.pairs[p].x : 0.0);
    f2 lpc = {0.f, 0.f}, lmc = {0.f, 0.f}, lpp = {0.f, 0.f}, lmp = {0.f, 0.f};
    int scp = 0, scm = 0;
    const float ulx = __int_as_float((127 - lexp) << 23);  // 1 / u_p
    float wfp = 0.f, wfm = 0.f;  // weight of the +s / -s values over u_p (zero until the pair joins)
    bool settled = false;        // every lane of the warp at scale 0 (warp-uniform)

    // 4 degrees from lb4 (lb4 - l0 even): digits of l+ / u_p and s l- / u_p packed per
    // pair of degrees into pk[set][digit][q / 2]; recursion advanced.  (Values of a
    // joined pair are not tested for negligibility: the join record already skips
    // the stretch before its first non-negligible degree pair, and later values
    // below the digits' grid give zero digits.)
    auto part = [&](int lb4, uint32_t (&pk)[NSET][kDig][2]) {
      float hold[NSET][kDig];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int l = lb4 + q;
        const bool odd = q & 1;
        float d[NSET][kDig];
        tca::split6(f2{lpc.h * wfp, lpc.l * wfp}, 98304.0f, d[0]);
        if (SPIN) {
          const float f = odd ? -wfm : wfm;
          tca::split6(f2{lmc.h * f, lmc.l * f}, 98304.0f, d[NSET - 1]);
        }
#pragma unroll
        for (int t = 0; t < NSET; ++t)
#pragma unroll
          for (int i = 0; i < kDig; ++i) {
            if (!odd) hold[t][i] = d[t][i];
            else pk[t][i][q >> 1] = tc::pack_bf16(hold[t][i], d[t][i]);
          }
        // recursion to l + 1 (past lmax the coefficients of lmax stand in: finite
        // values no output reads)
        const Coef32 cc = ld_coef32(cf + 2 * (l <= lmax ? l : lmax));
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
    };
    // the enhanced exponent's check after every block of 8 degrees (see mixed_common.cuh)
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
      if (lj <= lmax) {
        wfp = wfac(scp) * ulx;
        wfm = wfac(scm) * ulx;
      }
      settled = __all_sync(0xffffffffu, scp == 0 && scm == 0);
    };
    // this warp's digits of degrees 4h .. 4h + 3 of the block: entry tid % 8 of K-group
    // (set, tid / 8), N-group = digit, bytes 8h .. 8h + 7 of the 16-byte row
    auto store_b = [&](int h, const uint32_t (&pk)[NSET][kDig][2]) {
#pragma unroll
      for (int t = 0; t < NSET; ++t)
#pragma unroll
        for (int i = 0; i < kDig; ++i) {
          unsigned char *dst = Bbuf + i * S::B_SBO + (t * (tca::kPairs / 8) + tid / 8) * tca::kKStride + (tid % 8) * 16 + h * 8;
          *reinterpret_cast<uint2 *>(dst) = make_uint2(pk[t][i][0], pk[t][i][1]);
        }
    };
    // this warp's MMAs of a block into accumulator xb: one per K-step (16 entries:
    // two K-groups) of each set
    auto issue = [&](int xb) {
      tc::fence_after();
#pragma unroll
      for (int t = 0; t < NSET; ++t)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int kk = t * (tca::kPairs / 16) + 2 * warp + hh;
          const uint64_t ad = adesc0 + (uint64_t)((2 * kk * S::A_LBO) >> 4);
          const uint64_t bd = bdesc0 + (uint64_t)((2 * kk * tca::kKStride) >> 4);
          tc::mma_bf16(tbase + xb * tca::kDCols, ad, bd, idesc, 1u);
        }
      tc::mma_commit(&mine[warp]);
      tc::mma_commit(&full[xb]);
    };
    // reading warps: block ibp's D rows from accumulator ibp & 1 into shared memory;
    // the accumulator zeroed and released
    auto epi_read = [&](int ibp) {
      const int xb = ibp & 1;
      if (!wait_warp(&full[xb], (uint32_t)(ibp >> 1) & 1u)) {
        give_up();
        return;
      }
      tc::fence_after();
      const uint32_t ta = tlane + xb * tca::kDCols;
      uint32_t v[tca::kN / 16][16];
#pragma unroll
      for (int q = 0; q < tca::kN / 16; ++q) tc::tmem_ld16(ta + q * 16, v[q]);
      tc::tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < tca::kN / 16; ++q) tc::tmem_zero16(ta + q * 16);
      if (lane < S::EROWS) {
        float4 *er = reinterpret_cast<float4 *>(Ebuf + lane * tca::kEStride);
#pragma unroll
        for (int q = 0; q < tca::kN / 16; ++q)
#pragma unroll
          for (int r = 0; r < 4; ++r)
            er[4 * q + r] = make_float4(__uint_as_float(v[q][4 * r]), __uint_as_float(v[q][4 * r + 1]),
                                        __uint_as_float(v[q][4 * r + 2]), __uint_as_float(v[q][4 * r + 3]));
      }
      tc::tmem_wait_st();
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::bar_arrive(&freeb[xb]);
    };
    // the column and degree a lane sums: lanes 0 .. 15 of the reading warps, column
    // 2 warp + lane / 8, degree lane % 8; the slot entry it writes for block lbp
    // (nullptr: none; neg: add the negation)
    const int ocol = 2 * warp + (lane >> 3), odeg = lane & 7;
    const bool oact = warp < S::NREAD && lane < S::EROWS;
    auto out_at = [&](int lbp, bool &neg) -> double * {
      const int l = lbp + odeg, j = ocol >> 2, cc = ocol & 3;
      neg = false;
      if (!oact || l > lmax) return nullptr;
      if (SPIN) {
        neg = cc >= 2 && (odeg & 1);  // T2 = s (s T2)
        return outp + (int64_t)(l - l0) * V + 4 * j + cc;
      }
      // spin 0: the even-l columns at even l - l0, the odd ones at odd
      return (cc >> 1) == (odeg & 1) ? outp + (int64_t)(l - l0) * V + 2 * j + (cc & 1) : nullptr;
    };
    // the staged digit products of the lane's column and degree, by level: levels
    // 0 to 2 exact in FP32 (at most three sums of 2^22 quanta), added in
    // double-float; levels 3 to 6 in FP32; the slot entry written (prev: its value
    // from the group's earlier tiles)
    auto epi_sum = [&](double *o, bool neg, double prev) {
      if (o) {
        const float *e = Ebuf + (lane >> 3) * tca::kColRows * tca::kEStride + odeg;
        auto D = [&](int i, int j) { return e[j * tca::kEStride + i * 8]; };  // sum of G_j L_i
        const float L1 = __fadd_rn(D(1, 0), D(0, 1));
        const float L2 = __fadd_rn(__fadd_rn(D(2, 0), D(1, 1)), D(0, 2));
        float lo = 0.f;
#pragma unroll
        for (int k = 6; k >= 3; --k)
#pragma unroll
          for (int i = 0; i < kDig; ++i)
            if (k - i >= 0 && k - i < kDig) lo = __fadd_rn(lo, D(i, k - i));
        f2 t = two_sum(D(0, 0), L1);
        t = f2_add_lazy(t, f2{L2, 0.f});
        t = fast_two_sum(t.h, __fadd_rn(t.l, lo));
        const double val = f2_val(t);
        *o = prev + (neg ? -val : val);
      }
      __syncwarp();
    };

    int lb = lstart;
#pragma unroll 1
    for (; lb <= lmax; lb += tca::kBlk, ++ib) {
      const int xb = ib & 1;
      // the slot entry this lane adds the previous block to: read now, its latency
      // hidden behind this block's recursion
      bool neg_prev;
      double *const o_prev = lb > lstart ? out_at(lb - tca::kBlk, neg_prev) : nullptr;
      double prev = 0.0;
      if (o_prev && gi > 0) asm volatile("ld.global.f64 %0, [%1];" : "=d"(prev) : "l"(o_prev));
      if (lj == lb) {  // this pair joins: the recursion state where its terms start
        const JoinRec r = ld_join(jrec);
        lpc = r.lpc;
        lpp = r.lpp;
        lmc = r.lmc;
        lmp = r.lmp;
        scp = r.scp;
        scm = r.scm;
        wfp = wfac(scp) * ulx;
        wfm = wfac(scm) * ulx;
      }
      if (__any_sync(0xffffffffu, lj == lb)) settled = __all_sync(0xffffffffu, scp == 0 && scm == 0);
      // a warp none of whose pairs has joined adds nothing: no digits, no products,
      // a plain arrival.  Every warp first waits until the reading warps have
      // released the accumulator's previous block, so that no arrival (or commit)
      // of this block can fall into the phase of the block two before.
      const bool live = __any_sync(0xffffffffu, lj <= lb);
      if (live) {
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          uint32_t pk[NSET][kDig][2];
          part(lb + 4 * h, pk);
          // this warp's products of its previous block read the tiles: wait for them
          // before the first write (they have long finished by now)
          if (h == 0 && nmine > nmine_done) {
            if (!wait_warp(&mine[warp], (uint32_t)(nmine - 1) & 1u)) break;
            nmine_done = nmine;
          }
          store_b(h, pk);
        }
        if (nmine > nmine_done) {  // the wait above gave up
          give_up();
          break;
        }
        rescale();
        tc::fence_async_smem();
        __syncwarp();
      }
      if (ib >= 2 && !wait_warp(&freeb[xb], (uint32_t)((ib - 2) >> 1) & 1u)) {
        give_up();
        break;
      }
      if (live) {
        if (lane == 0) issue(xb);
        __syncwarp();
        ++nmine;
      } else if (lane == 0) {
        tc::bar_arrive(&full[xb]);
      }
      if (warp < S::NREAD && lb > lstart) {
        epi_read(ib - 1);
        if (!ok) break;
        epi_sum(o_prev, neg_prev, prev);
      }
    }
    if (!ok) continue;  // to the next tile's barrier, where the CTA stops
    if (warp < S::NREAD) {  // the tile's last block
      bool neg;
      double *o = out_at(lb - tca::kBlk, neg);
      const double prev = (o && gi > 0) ? *o : 0.0;
      epi_read(ib - 1);
      if (!ok) continue;
      epi_sum(o, neg, prev);
    }
  }

  // leave: flag a wait that gave up, let this warp's products in flight finish
  // (bounded), release TMEM
  if (!ok && tid == 0) atomicOr(ta.err, 1);
  if (nmine > nmine_done) tc::bar_wait(&mine[warp], (uint32_t)(nmine - 1) & 1u);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tbase, 2 * tca::kDCols);
}

template <int NJ, bool SPIN>
__global__ void __launch_bounds__(tca::kPairs, (tca::AnaShape<NJ, SPIN>::MINB)) tc_ana(TcArgs ta) {
  extern __shared__ __align__(128) unsigned char tca_smem[];
  tc_ana_body<NJ, SPIN>(ta, ta.m.ana_items[blockIdx.x], tca_smem);
}

// batches: item (mi, first tile, slot << 8 | tiles, record); the record holds the plan's arguments
template <int NJ, bool SPIN>
__global__ void __launch_bounds__(tca::kPairs, (tca::AnaShape<NJ, SPIN>::MINB))
    tc_ana_batch(const TcArgs *__restrict__ args, const int4 *__restrict__ items) {
  extern __shared__ __align__(128) unsigned char tca_smem[];
  const int4 it = items[blockIdx.x];
  tc_ana_body<NJ, SPIN>(args[it.w], make_int4(it.x, it.y, it.z, 0), tca_smem);
}

template <int NJ, bool SPIN>
static cudaError_t tca_set_smem() {
  cudaError_t e = cudaSuccess;
  for (const void *k : {(const void *)tc_ana<NJ, SPIN>, (const void *)tc_ana_batch<NJ, SPIN>}) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, tca::AnaShape<NJ, SPIN>::SMEM_LAUNCH);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  }
  return e;
}

cudaError_t tc_ana_prepare_device() {
  cudaError_t e = tca_set_smem<1, false>();
  if (e == cudaSuccess) e = tca_set_smem<2, false>();
  if (e == cudaSuccess) e = tca_set_smem<1, true>();
  if (e == cudaSuccess) e = tca_set_smem<2, true>();
  return e;
}

bool tc_ana_supported(int spin, int njobs_pad) {
  (void)spin;
  return njobs_pad <= 2;
}

cudaError_t launch_leg_tc_ana_batch(int spin, int nj, const void *targs, const int4 *items, int n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const TcArgs *a = static_cast<const TcArgs *>(targs);
  if (spin == 0) {
    switch (nj) {
      case 1: tc_ana_batch<1, false><<<n, tca::kPairs, tca::AnaShape<1, false>::SMEM_LAUNCH, st>>>(a, items); break;
      case 2: tc_ana_batch<2, false><<<n, tca::kPairs, tca::AnaShape<2, false>::SMEM_LAUNCH, st>>>(a, items); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (nj) {
      case 1: tc_ana_batch<1, true><<<n, tca::kPairs, tca::AnaShape<1, true>::SMEM_LAUNCH, st>>>(a, items); break;
      case 2: tc_ana_batch<2, true><<<n, tca::kPairs, tca::AnaShape<2, true>::SMEM_LAUNCH, st>>>(a, items); break;
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_leg_tc_ana(const sht_plan_s *P, const void *mixargs, int n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  TcArgs ta;
  memcpy(&ta.m, mixargs, sizeof(MixArgs));
  ta.lam_bound = P->tc_lam_bound;
  ta.err = P->d_err;
  const int nj = P->njobs_pad;
  if (P->spin == 0) {
    switch (nj) {
      case 1: tc_ana<1, false><<<n, tca::kPairs, tca::AnaShape<1, false>::SMEM_LAUNCH, st>>>(ta); break;
      case 2: tc_ana<2, false><<<n, tca::kPairs, tca::AnaShape<2, false>::SMEM_LAUNCH, st>>>(ta); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (nj) {
      case 1: tc_ana<1, true><<<n, tca::kPairs, tca::AnaShape<1, true>::SMEM_LAUNCH, st>>>(ta); break;
      case 2: tc_ana<2, true><<<n, tca::kPairs, tca::AnaShape<2, true>::SMEM_LAUNCH, st>>>(ta); break;
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

}  // namespace sht
