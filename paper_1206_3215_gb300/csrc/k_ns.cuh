// Fused passes of the Navier-Stokes Crank-Nicolson / fixed-point scheme
// (vorticity form, Section 3.3; time stepping, Section 4.3).
//
//   (w^{k+1} - w^n)/dt - nu Lap (w^{k+1} + w^n)/2 + (J^k + J^n)/2 = 0,
//   J = psi_y w_x - psi_x w_y,  Lap psi = -w,
// iterated over k until integral (w^{k+1} - w^k)^2 < tol.  The implicit
// midpoint variant replaces (J^k + J^n)/2 by J^k_mid, the Jacobian of
// (w^k + w^n)/2: the column pass then transforms the derivatives of that
// midpoint instead of those of w^{k+1}, and J_hat^n is not kept.  Its first
// update (w^0 = w^n) is the same as Crank-Nicolson's.
//
// The Jacobian needs four derivative fields; they are packed into two complex
// fields whose transforms are
//   C1 = psi_y - i psi_x  <->  (kx + i ky) psi_hat,
//   C2 = w_x + i w_y      <->  i (kx + i ky) w_hat,
// so that J = Re C1 Re C2 + Im C1 Im C2 pointwise.  One fixed-point update is
// a row pass (row inverse transforms of C1 and C2, J, row forward transform)
// and a column pass (column forward transform -> J_hat with the 2/3 mask, CN
// update, FP64 partial of |w^{k+1} - w^k|^2, derivatives of w^{k+1}, column
// inverse transforms into C1 and C2).  A small kernel then folds the partials
// per field in a fixed order and decides, per field, whether to stop.
//
// Vorticity iterates live in three buffers per field: w^n in buffer idx, the
// iterate of update k >= 1 in (idx + 1 + ((k - 1) & 1)) % 3.  Fields that have
// converged skip their loads and stores while the others iterate, so a field
// gets exactly the updates it would get alone.
#pragma once
#include "launch.cuh"

namespace pss {

// The NS column and derivative passes keep one array of P points per thread
// live at a time: the column pass rebuilds the second derivative field from
// the iterate it has just stored.  With every transform of a pass running
// through one forward-FFT body (F^-1 x = conj(F conj x), exact) they fit the
// lean shape (one buffer, <= 128 registers) with 32 points per thread (the
// derivative pass takes 16 from 1024 on, where 32 spills).  Measured at
// 4096^2 FP32: column pass 1.23 -> 0.82 ms per update in the lean shape with
// 16 points, 0.54 -> 0.51 ms with 32 points (wider tiles) after the 2/3
// pruning.
#ifndef NS_PMAX
#define NS_PMAX 32
#endif
#ifndef NS_PMAX_BIG
#define NS_PMAX_BIG 32
#endif
#ifndef NS_PREP_PMAX_BIG
#define NS_PREP_PMAX_BIG 16
#endif
__host__ __device__ constexpr int ns_pmax(int n) { return n <= 1024 ? NS_PMAX : NS_PMAX_BIG; }
#ifndef NS_LEAN
#define NS_LEAN true
#endif

// correctly rounded reciprocal (the value 1 / x rounds to, without the
// division's instruction sequence)
__device__ __forceinline__ float ns_rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double ns_rcp(double x) { return __drcp_rn(x); }

struct NsField {
    int idx;        // buffer holding w^n
    int active;     // still iterating in this step
    int nonconv;    // reached max_iter in some step (sticky)
    int pad;
    long long updates;  // CN updates (= Jacobian evaluations) summed over steps
};

__host__ __device__ __forceinline__ int ns_buf(int idx, int k)
{
    return k == 0 ? idx : (idx + 1 + ((k - 1) & 1)) % 3;
}

// Products and fused multiply-adds with their roundings written out: the
// column pass's arithmetic is inlined into several kernels (one-part and
// split passes, per-point staging), and a compiler free to contract a * b + c
// may fuse a different product in each; with these they agree bit for bit.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// packed derivative spectra of w_hat at wavenumber (kx, ky) (odd-derivative
// wavenumbers: zero at the Nyquist index), times the inverse-transform scale:
// which = 0: C1 = (kx + i ky) psi_hat, psi_hat = w_hat / |k|^2 (0 at k = 0);
// which = 1: C2 = i (kx + i ky) w_hat
template <class V, class R> __device__ __forceinline__ V ns_deriv(int which, V w, R kx, R ky, R k2, R s)
{
    if (which == 0) {
        const R inv = k2 > R(0) ? s / k2 : R(0);
        const V p{mul_rn(w.x, inv), mul_rn(w.y, inv)};  // psi_hat * s
        return V{fma_rn(kx, p.x, -mul_rn(ky, p.y)), fma_rn(kx, p.y, mul_rn(ky, p.x))};
    }
    return V{mul_rn(-fma_rn(kx, w.y, mul_rn(ky, w.x)), s), mul_rn(fma_rn(kx, w.x, -mul_rn(ky, w.y)), s)};
}

// The row pass keeps both inputs in registers (measured at 4096^2: 0.22 ms
// with 16 points per thread, double buffer and up to 255 registers, against
// 0.34 ms in the lean shape with the C1 row parked in shared memory)
template <class Rl> struct NsRow {
    static constexpr int NIN = 2;
    static constexpr bool LEAN = false;
    static constexpr int PMAX = 16;
    V2<Rl> *c1, *c2;  // in: C1, C2 rows; out: row transform of J into c1
    const NsField *fs;
    int lgy;      // log2 ny: row r belongs to field r >> lgy
    int dealias;  // 2/3 rule: columns with 3 |mx| >= nx are not written (they stay
                  // zero: the column pass skips them and the mask discards J there)
    int half;     // half spectra: only columns 0 .. nx/2 of J are read, so only they are written
    __device__ const V2<Rl> *in(int k) const { return k == 0 ? c1 : c2; }
    template <int N, int P, int BLOCK, class Sm>
    __device__ __forceinline__ void row(V2<Rl> (&v)[2][P], int64_t r, bool ok, int t, const Sm (&sm)[2],
                                        const TW<Rl> *tw) const
    {
        block_fft<N, P, +1, BLOCK>(v[0], sm[0], t, tw);
        block_fft<N, P, +1, BLOCK>(v[1], sm[1], t, tw);
        fence(v[0]);
        fence(v[1]);
#pragma unroll
        for (int m = 0; m < P; ++m) v[0][m] = V2<Rl>{v[0][m].x * v[1][m].x + v[0][m].y * v[1][m].y, Rl(0)};
        fence(v[0]);
        block_fft<N, P, -1, BLOCK>(v[0], sm[0], t, tw);
        const bool live = ok && fs[r >> lgy].active;
        constexpr int T = N / P;
        V2<Rl> *p = c1 + r * N + t;
#pragma unroll
        for (int m = 0; m < P; ++m, p += T) {
            const int x = t + T * m;
            const bool kept = (!dealias || 3 * (x < N / 2 ? x : N - x) < N) && (!half || x <= N / 2);
            if (live && kept) *p = v[0][m];
        }
    }
};

// Column pass of one fixed-point update.  HALF: the vorticity iterates and
// J_hat^n are half spectra (columns kx = 0 .. nxf/2 of rows of stride nx),
// J and C1, C2 stay full-width rows (stride nxf = in_stride); each visited
// column kx writes the derivative fields at kx and at nxf - kx (the
// transforms of a real field at -kx are the conjugates of those at kx, with
// the spectrum taken at -kx), so four inverse transforms per column replace
// two on twice as many columns.
// Squared difference d^2 added to the double-float accumulator (hi, lo) in
// FP32 arithmetic: d^2 = p + e exactly (e by a fused multiply-add), p enters
// hi by Knuth's two-sum and the rounding errors collect in lo.  The sum keeps
// about twice the FP32 precision without the FP64 pipe, which on GB300 runs
// 64 times slower than FP32 and held up the column pass.
__device__ __forceinline__ void df_add_sq(float &hi, float &lo, float d)
{
    const float p = __fmul_rn(d, d);  // rounded on its own: the sum below must not fuse it
    const float e = __fmaf_rn(d, d, -p);
    const float sum = hi + p;
    const float bp = sum - hi;
    const float err = (hi - (sum - bp)) + (p - bp);
    hi = sum;
    lo += err + e;
}

template <class Rl, bool MID, bool HALF = false> struct NsCol {
    static constexpr int NIN = 1;
    static constexpr bool COL_LAND = true;  // exchanges and the norm partial sync per tile (BLOCK)
    // half spectra, one-buffer shapes (4096 points and more): each tile runs
    // in two parts (k_col_split), the update with C1's two outputs and C2's
    // two outputs.  Measured at 4096^2 (column pass per update, CN): batch 1
    // 351 -> 299 us, batch 2 587 -> 504 us; with full spectra, where the
    // second part is one transform, 307 -> 318 us, so those stay in one part
    static constexpr bool COL_SPLIT = HALF;
    static constexpr bool LEAN = NS_LEAN;
    static constexpr int PMAX = NS_PMAX;
    static constexpr int NOUT = HALF ? 4 : 2;  // inverse transforms per column
    __host__ __device__ static constexpr int pmax(int n) { return ns_pmax(n); }
    V2<Rl> *c1, *c2;        // in: J row transforms (c1); out: C1, C2 of w^{k+1}
    V2<Rl> *w0, *w1, *w2;   // vorticity buffers
    V2<Rl> *jn;             // J_hat^n (written when k == 0)
    NsField *fs;
    double *partials;       // [field][column group]
    const Rl *kxo, *kyo, *kx2, *ky2, *keepx, *keepy;
    Rl half_dt, half_dt_nu, inv_n2;
    int64_t nx;             // row stride of w and J_hat^n (half spectra: nxf/2 + 8)
    const int *kptr;  // fixed-point update index of this pass (device, set by k_ns_advance)
    int W;
    int64_t in_stride;      // row stride of J, C1, C2 (= nxf)
    // 2/3 rule: column groups skip_lo .. skip_lo + skip_n - 1 hold only modes
    // with 3|mx| >= nx, which the mask keeps at zero in w, J and the
    // derivative fields; the pass does not visit them (0, 0 without dealiasing)
    int64_t skip_lo, skip_n;
    int *status;  // set when a tile copy did not arrive
    // split column pass (k_col_split): item counter (zero at launch), epoch of
    // this pass (the published value is *epoch + 1), per-tile done words
    int *claim;
    const int *epoch;
    unsigned *tile_done;
    static constexpr bool midpoint = MID;  // implicit midpoint, else trapezoidal Jacobian
    __host__ __device__ const V2<Rl> *in(int) const { return c1; }
    __device__ V2<Rl> *wb(int b) const { return b == 0 ? w0 : b == 1 ? w1 : w2; }
    // field whose derivatives feed the next Jacobian: w^{k+1}, or the
    // midpoint (w^{k+1} + w^n)/2
    __device__ __forceinline__ V2<Rl> jfield(V2<Rl> w1v, V2<Rl> a_n) const
    {
        if constexpr (MID) return V2<Rl>{mul_rn(Rl(0.5), w1v.x + a_n.x), mul_rn(Rl(0.5), w1v.y + a_n.y)};
        return w1v;
    }
    template <int N, int P, int BLOCK, class Sm>
    __device__ __forceinline__ void col(V2<Rl> (&vv)[1][P], int64_t field, int x, int t,
                                        const Sm (&sm)[1], const TW<Rl> *tw) const
    {
        col_range<N, P, BLOCK>(vv[0], field, x, t, sm[0], tw, 0, NOUT);
    }
    // the two parts of a tile in the split column pass (k_col_split): part 0
    // the update and the outputs of C1, part 1 those of C2, rebuilt from the
    // iterate part 0 stored
    template <int N, int P, int BLOCK, class Sm>
    __device__ __forceinline__ void col_part(V2<Rl> (&vv)[1][P], int64_t field, int x, int t,
                                             const Sm (&sm)[1], const TW<Rl> *tw, int part) const
    {
        col_range<N, P, BLOCK>(vv[0], field, x, t, sm[0], tw, part ? NOUT / 2 : 0, part ? NOUT : NOUT / 2);
    }
    // outputs o0 .. o1 - 1 of the column (o0 = 0: v holds the staged column of
    // J; the update comes first and the partial of the norm is written)
    template <int N, int P, int BLOCK, class Sm>
    __device__ __forceinline__ void col_range(V2<Rl> (&v)[P], int64_t field, int x, int t, const Sm &sm,
                                              const TW<Rl> *tw, int o0, int o1) const
    {
        constexpr int T = N / P;
        const int k = *kptr;
        const NsField f = fs[field];
        const int64_t nxf = in_stride;
        // half spectra: the padding columns beyond nxf/2 carry nothing
        const bool valid = !HALF || 2 * int64_t(x) <= nxf;
        const bool live = f.active != 0 && valid;
        const int64_t base = field * N * nx + x;
        const V2<Rl> *wn = wb(f.idx) + base;
        const V2<Rl> *wk = wb(ns_buf(f.idx, k)) + base;
        V2<Rl> *wk1 = wb(ns_buf(f.idx, k + 1)) + base;
        const int xs = valid ? x : 0;  // table index (the padding reads column 0's entries)
        const Rl kx = __ldg(kxo + xs), kxx = __ldg(kx2 + xs), mx = __ldg(keepx + xs);
        double acc = 0.0;
        float acc_hi = 0.0f, acc_lo = 0.0f;  // FP32: double-float partial of this thread
        if (f.active && o0 == 0) {  // the update reads w^n, w^k (and J_hat^n) after the forward transform
            // by row: thread i of the tile's T W threads asks for rows i, i + T W, ...
            // (one 32-byte row segment of the tile per request)
            const int64_t tb = field * N * nx + (x - x % W);
#pragma unroll
            for (int r = t * W + x % W; r < N; r += T * W) {
                const int64_t o = tb + int64_t(r) * nx;
                prefetch_l2(wb(f.idx) + o);
                prefetch_l2(wb(ns_buf(f.idx, k)) + o);
                if (!MID && k > 0) prefetch_l2(jn + o);
            }
        }
        // pass 0: J_hat and the update; pass p > 0: output p - 1, a derivative
        // field of the new iterate (or of the midpoint), inverse transformed
        // through the forward body.  Pass 0 leaves the field of output 0 in
        // v; every later one is rebuilt from the iterate stored in pass 0
        // (loads that bypass L1: part 1 of the split pass may run on another
        // SM than the part that stored it)
#pragma unroll 1
        for (int pass = o0 == 0 ? 0 : o0 + 1; pass <= o1; ++pass) {
            if (pass >= 2) {
                const int out = pass - 1;
                const int nwhich = HALF ? out >> 1 : out;
                const bool nmirror = HALF && (out & 1);
                const Rl sx = nmirror ? -kx : kx;
                // at -kx a field's transform is conj(IFFT(conj(d(-kx, -ky)) w_hat(kx, ky))):
                // d(-kx, ky) itself for C1, its negative for C2 = i (kx + i ky) w_hat
                const Rl sg = (nmirror && nwhich == 1) ? Rl(-1) : Rl(1);
#pragma unroll
                for (int m = 0; m < P; ++m) {
                    const int y = t + T * m;
                    const int64_t o = int64_t(y) * nx;
                    const V2<Rl> w1v = live ? __ldcg(wk1 + o) : V2<Rl>{0, 0};
                    const V2<Rl> a_n = (MID && live) ? ld_stream(wn + o) : V2<Rl>{0, 0};
                    const V2<Rl> d = ns_deriv(nwhich, jfield(w1v, a_n), sx, __ldg(kyo + y), kxx + __ldg(ky2 + y),
                                              inv_n2);
                    v[m] = V2<Rl>{sg * d.x, sg * d.y};
                }
            }
            if (pass > 0) conj_all(v);
            block_fft<N, P, -1, BLOCK>(v, sm, t, tw);
            if (pass == 0) {
                // loads of CH points ahead of their stores (the buffers may alias
                // as far as the compiler knows, so it would not reorder them)
                constexpr int CH = 4;
                V2<Rl> ln[CH], lk[CH], lj[CH];
#pragma unroll
                for (int m = 0; m < P; ++m) {
                    const int y = t + T * m;
                    const int64_t o = int64_t(y) * nx;
                    if (m % CH == 0)
#pragma unroll
                        for (int c = 0; c < CH && m + c < P; ++c) {
                            const int64_t oc = int64_t(t + T * (m + c)) * nx;
                            ln[c] = live ? ld_stream(wn + oc) : V2<Rl>{0, 0};
                            lk[c] = live ? ld_stream(wk + oc) : V2<Rl>{0, 0};
                            if (!MID && k > 0) lj[c] = live ? ld_stream(jn + base + oc) : V2<Rl>{0, 0};
                        }
                    const Rl mask = mul_rn(mx, __ldg(keepy + y));
                    const V2<Rl> jk{mul_rn(v[m].x, mask), mul_rn(v[m].y, mask)};
                    // midpoint: jk is already J((w^k + w^n)/2), used twice below
                    V2<Rl> jnv = jk;
                    if constexpr (!MID) {
                        if (k == 0) {
                            if (live) jn[base + o] = jk;
                        } else {
                            jnv = live ? lj[m % CH] : jk;
                        }
                    }
                    const V2<Rl> a_n = ln[m % CH];
                    const V2<Rl> a_k = lk[m % CH];
                    const Rl kk = kxx + __ldg(ky2 + y);
                    // w^{k+1} = [(1 - a) w^n - dt/2 (J^k + J^n)] / (1 + a), a = dt nu |k|^2 / 2,
                    // formed as w^n minus a small increment so that FP32 rounds
                    // the increment, not the nearly-unit decay factor, every step
                    const Rl a = mul_rn(half_dt_nu, kk);
                    const Rl inv = ns_rcp(Rl(1) + a);  // correctly rounded, as 1 / (1 + a)
                    const Rl a2 = Rl(2) * a;           // exact
                    const V2<Rl> inc{mul_rn(fma_rn(a2, a_n.x, mul_rn(half_dt, jk.x + jnv.x)), inv),
                                     mul_rn(fma_rn(a2, a_n.y, mul_rn(half_dt, jk.y + jnv.y)), inv)};
                    const V2<Rl> w1v{a_n.x - inc.x, a_n.y - inc.y};
                    if constexpr (sizeof(Rl) == 4) {
                        // w^{k+1} - w^k: exact in FP32 once the iterates agree to a
                        // factor of two (Sterbenz), one rounding before that
                        if (valid) {
                            df_add_sq(acc_hi, acc_lo, w1v.x - a_k.x);
                            df_add_sq(acc_hi, acc_lo, w1v.y - a_k.y);
                        }
                    } else {
                        const double ex = double(w1v.x) - double(a_k.x), ey = double(w1v.y) - double(a_k.y);
                        if (valid) acc += ex * ex + ey * ey;
                    }
                    if (live) wk1[o] = w1v;
                    v[m] = ns_deriv(0, jfield(w1v, a_n), kx, __ldg(kyo + y), kk, inv_n2);
                }
            } else {
                // output pass - 1: C1 or C2, at kx or (half spectra) mirrored at nxf - kx
                const int out = pass - 1;
                const int which = HALF ? out >> 1 : out;
                const bool mirror = HALF && (out & 1);
                if (!mirror) conj_all(v);  // the mirrored column stores the conjugate
                const bool dup = mirror && (x == 0 || 2 * int64_t(x) == nxf);
                V2<Rl> *dst = (which == 0 ? c1 : c2) + field * N * nxf + (mirror ? nxf - x : x);
                store_line<P, T>(v, dst, nxf, t, live && !dup);
            }
        }
        if (o0 == 0) {
            // FP64 partial of |w^{k+1} - w^k|^2 over this tile, folded in a fixed order
            const int64_t g = x / W;
            if constexpr (sizeof(Rl) == 4) acc = double(acc_hi) + double(acc_lo);
            block_partial<BLOCK>(acc, partials + field * (nx / W - skip_n) + (g < skip_lo ? g : g - skip_n));
        }
    }
    // sum over the threads of the tile in a fixed tree; the tile's first
    // thread writes.  BLOCK <= 1: the tile is the CTA; BLOCK > 1: a group of
    // BLOCK threads of a CTA that holds two tiles (its own named barrier, its
    // own warps' slots)
    template <int BLOCK> __device__ __forceinline__ void block_partial(double acc, double *out) const
    {
        __shared__ double red[32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if constexpr (BLOCK > 1) {
            fft_sync<BLOCK>();
            if (lane == 0) red[warp] = acc;
            fft_sync<BLOCK>();
            if (threadIdx.x % BLOCK == 0) {
                double s = 0.0;
                for (int i = 0; i < BLOCK / 32; ++i) s += red[warp + i];
                *out = s;
            }
        } else {
            __syncthreads();
            if (lane == 0) red[warp] = acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                double s = 0.0;
                for (int i = 0; i < int((blockDim.x + 31) >> 5); ++i) s += red[i];
                *out = s;
            }
        }
    }
};

// derivatives of w^n into C1, C2: the state after set_state (every field's
// w^n in buffer 0: fs == nullptr), and, for the midpoint scheme, at the start
// of every step (w^n in buffer fs[field].idx), since its last column pass
// leaves the derivatives of the midpoint rather than those of w^{n+1}
template <class Rl, bool HALF = false> struct NsPrep {
    static constexpr int NIN = 1;
    static constexpr bool LEAN = NS_LEAN;
    static constexpr int PMAX = NS_PMAX;
    static constexpr int NOUT = HALF ? 4 : 2;
    __host__ __device__ static constexpr int pmax(int n) { return n < 1024 ? NS_PMAX : NS_PREP_PMAX_BIG; }
    const V2<Rl> *w0, *w1, *w2;
    const NsField *fs;
    V2<Rl> *c1, *c2;
    const Rl *kxo, *kyo, *kx2, *ky2;
    Rl inv_n2;
    int64_t nx;   // row stride of w (half spectra: nxf/2 + 8)
    int64_t nxf;  // row stride of C1, C2
    __device__ const V2<Rl> *in(int, int64_t field) const
    {
        const int b = fs ? fs[field].idx : 0;
        return b == 0 ? w0 : b == 1 ? w1 : w2;
    }
    template <int N, int P, int BLOCK, class Sm>
    __device__ __forceinline__ void col(V2<Rl> (&vv)[1][P], int64_t field, int x, int t,
                                        const Sm (&sm)[1], const TW<Rl> *tw) const
    {
        constexpr int T = N / P;
        V2<Rl>(&v)[P] = vv[0];
        const int64_t base = field * N * nx + x;
        const V2<Rl> *w = in(0, field) + base;
        const bool valid = !HALF || 2 * int64_t(x) <= nxf;
        const int xs = valid ? x : 0;
        const Rl kx = __ldg(kxo + xs), kxx = __ldg(kx2 + xs);
        // the first output from the staged column, the others from the column
        // re-read; half spectra: C1, C2 at kx and mirrored at nxf - kx
#pragma unroll 1
        for (int out = 0; out < NOUT; ++out) {
            const int which = HALF ? out >> 1 : out;
            const bool mirror = HALF && (out & 1);
            if (out > 0)
#pragma unroll
                for (int m = 0; m < P; ++m) v[m] = w[int64_t(t + T * m) * nx];
            const Rl sx = mirror ? -kx : kx;
            const Rl sg = (mirror && which == 1) ? Rl(-1) : Rl(1);  // as in NsCol
#pragma unroll
            for (int m = 0; m < P; ++m) {
                const int y = t + T * m;
                const V2<Rl> d = ns_deriv(which, v[m], sx, __ldg(kyo + y), kxx + __ldg(ky2 + y), inv_n2);
                v[m] = V2<Rl>{sg * d.x, sg * d.y};
            }
            conj_all(v);
            block_fft<N, P, -1, BLOCK>(v, sm[0], t, tw);
            if (!mirror) conj_all(v);
            const bool dup = mirror && (x == 0 || 2 * int64_t(x) == nxf);
            V2<Rl> *dst = (which == 0 ? c1 : c2) + field * N * nxf + (mirror ? nxf - x : x);
            store_line<P, T>(v, dst, nxf, t, valid && !dup);
        }
    }
};

// Column groups (w columns each, of a row of stride sx) the column pass
// skips, as one run [lo, lo + n): with full spectra the groups whose every
// column has 3 |mx| >= nxf (dealiasing only); with half spectra the groups
// whose columns all have 2x > nxf (padding) or, dealiasing, 3x >= nxf.
inline void ns_skip_groups(int64_t nxf, int64_t sx, int w, bool half, bool dealias, int64_t *lo, int64_t *n)
{
    auto skipped = [&](int64_t x) {
        if (half) return 2 * x > nxf || (dealias && 3 * x >= nxf);
        return dealias && 3 * (x < nxf / 2 ? x : nxf - x) >= nxf;
    };
    int64_t first = -1, last = -1;
    for (int64_t g = 0; g < sx / w; ++g) {
        bool all = true;
        for (int64_t x = g * w; x < (g + 1) * w; ++x) all = all && skipped(x);
        if (all) {
            if (first < 0) first = g;
            last = g;
        }
    }
    *lo = first < 0 ? 0 : first;
    *n = first < 0 ? 0 : last - first + 1;
}

// column pass of one fixed-point update (scheme chosen by MID, layout by
// HALF); nxf is the grid's row length, sx the row stride of w and J_hat^n
template <class Rl, bool MID, bool HALF>
cudaError_t ns_col_run(V2<Rl> *c1, V2<Rl> *c2, V2<Rl> *const w[3], V2<Rl> *jn, void *fs, double *partials,
                        const Rl *kxo, const Rl *kyo, const Rl *kx2, const Rl *ky2, const Rl *keepx,
                        const Rl *keepy, double dt, double nu, int64_t nxf, int64_t sx, int64_t ny, int64_t batch,
                        const int *ctl, const TW<Rl> *twy, int *groups_out, cudaStream_t s, bool dealias)
{
    using Op = NsCol<Rl, MID, HALF>;
    Op op{c1, c2, w[0], w[1], w[2], jn, static_cast<NsField *>(fs), partials, kxo, kyo, kx2, ky2,
          keepx, keepy, Rl(0.5 * dt), Rl(0.5 * dt * nu), Rl(1.0 / (double(nxf) * double(ny))), sx, ctl, 0,
          nxf, 0, 0, const_cast<int *>(ctl) + FLAG_SLOT_PASS_STATUS, const_cast<int *>(ctl) + FLAG_SLOT_SPLIT_CLAIM,
          ctl + FLAG_SLOT_EPOCH, reinterpret_cast<unsigned *>(const_cast<int *>(ctl) + FLAG_TILE_DONE)};
    switch (ny) {
#define PSS_CASE(N)                                                                          \
    case N:                                                                                  \
        op.W = ColCfgOf<Rl, N, Op>::W;                                                       \
        if (sx % op.W) return cudaErrorInvalidValue;                                         \
        ns_skip_groups(nxf, sx, op.W, HALF, dealias, &op.skip_lo, &op.skip_n);               \
        *groups_out = int(sx / op.W - op.skip_n);                                            \
        return launch_col_n<Rl, N>(op, twy, sx, batch, s);
        PSS_FOR_EACH_N(PSS_CASE)
#undef PSS_CASE
    default: return cudaErrorInvalidValue;
    }
}

// the other instantiations live in their own translation units: midpoint on
// full spectra (k_ns_mid.cu), both schemes on half spectra (k_ns_half.cu)
template <class Rl>
cudaError_t ns_col_mid(V2<Rl> *c1, V2<Rl> *c2, V2<Rl> *const w[3], V2<Rl> *jn, void *fs, double *partials,
                       const Rl *kxo, const Rl *kyo, const Rl *kx2, const Rl *ky2, const Rl *keepx,
                       const Rl *keepy, double dt, double nu, int64_t nx, int64_t ny, int64_t batch,
                       const int *ctl, const TW<Rl> *twy, int *groups_out, cudaStream_t s, bool dealias);
template <class Rl>
cudaError_t ns_col_half(V2<Rl> *c1, V2<Rl> *c2, V2<Rl> *const w[3], V2<Rl> *jn, void *fs, double *partials,
                        const Rl *kxo, const Rl *kyo, const Rl *kx2, const Rl *ky2, const Rl *keepx,
                        const Rl *keepy, double dt, double nu, int64_t nxf, int64_t sx, int64_t ny, int64_t batch,
                        const int *ctl, int midpoint, const TW<Rl> *twy, int *groups_out, cudaStream_t s,
                        bool dealias);
template <class Rl>
cudaError_t ns_prep_half(V2<Rl> *const w[3], const void *fs, V2<Rl> *c1, V2<Rl> *c2, const Rl *kxo, const Rl *kyo,
                         const Rl *kx2, const Rl *ky2, int64_t nxf, int64_t sx, int64_t ny, int64_t batch,
                         const TW<Rl> *twy, cudaStream_t s);

}  // namespace pss
