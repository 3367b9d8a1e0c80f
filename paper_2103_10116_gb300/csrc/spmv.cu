// spmv.cu -- sparse matrix-vector product kernels for sm_103a.
//
// y = A x (Section 5 of arXiv 2103.10116 defines SpMV and the CSR / COO
// layouts; ELL and HYB are this library's additional storage orders).
//
// GB300 shapes the design in one way above all: IEEE double FMA throughput is
// low (about 2 FMA per SM per clock), so an FP64 SpMV that streams 12 bytes
// per nonzero from HBM is co-bound by the FP64 pipe.  Every FP64 kernel here
// therefore spends exactly one FMA per stored entry and as few extra FP64
// instructions as it can: rows are accumulated sequentially by one thread
// (merge-path CSR, ELL, segmented COO) and warp-shuffle reductions are kept
// for the classic vector kernel only.
//
// Determinism: no floating-point atomics.  Rows that straddle a thread or tile
// boundary are completed by a fixed-order carry chain; the per-tile carries
// and the dot-product partials are finished by the last block to arrive, in
// index order, so every run gives the same bits.
#include <climits>
#include <map>
#include <mutex>
#include <utility>

#include "dev_common.cuh"
#include "kstate.cuh"
#include "spx_internal.cuh"

namespace spx {

// ------------------------------------------------------------------ epilogue helpers
template <class T> __device__ __forceinline__ bool is_one(T a)
{
    if constexpr (sizeof(T) == 8) return __double_as_longlong(a) == 0x3FF0000000000000LL;
    else return __float_as_int(a) == 0x3F800000;
}

template <class T> __device__ __forceinline__ T epi_val(const Epi<T> &e, int64_t r, T t)
{
    if (!is_one(e.alpha)) t *= e.alpha;
    if (e.z) t = fma(e.beta, e.z[r], t);
    return t;
}

template <class T>
__device__ __forceinline__ void final_write(const Epi<T> &e, int64_t r, T t, T &d0, T &d1)
{
    const T v = epi_val(e, r, t);
    e.y[r] = v;
    if (e.w) d0 = fma(e.w[r], v, d0);
    if (e.want_yy) d1 = fma(v, v, d1);
}

// Row output.  MODE 0: the general epilogue; 1: plain store y = t; 2: y +=
// alpha t (the COO part of HYB); 3: y += t.  The row-block, nnz-split and ELL
// kernels also take the Krylov solvers' epilogues as modes of their own: 4:
// y = t with w.y (CG's
// q = A p with p.q, BiCGSTAB's and CGS's v = A p with r^.v); 5: the same and
// y.y (BiCGSTAB's t = A s with t.s, t.t); 6: y = t with y.y (GMRES's A v);
// 7: y = z - t with y.y (the residual b - A x).  Fixing the mode at compile
// time keeps the unused epilogue terms out of the row-emission code:
// predicated-off FP64 instructions still take FP64 issue slots, and the FP64
// pipe is what bounds these kernels.  Every mode rounds as MODE 0 does.
template <int MODE, class T>
__device__ __forceinline__ void out_row(const Epi<T> &e, int64_t r, T t, T &d0, T &d1)
{
    if constexpr (MODE == 0) final_write(e, r, t, d0, d1);
    else if constexpr (MODE == 1) e.y[r] = t;
    else if constexpr (MODE >= 4) {
        const T v = MODE == 7 ? fma(T(1), e.z[r], -t) : t;
        e.y[r] = v;
        if constexpr (MODE == 4 || MODE == 5) d0 = fma(e.w[r], v, d0);
        if constexpr (MODE >= 5) d1 = fma(v, v, d1);
    }
    // add modes: one add per row into a y no other thread touches in this launch,
    // so a fire-and-forget atomic gives the same bits as load + store without
    // stalling the emitting lane on the load
    else if constexpr (MODE == 2) atomicAdd(e.y + r, e.alpha * t);
    else atomicAdd(e.y + r, t);
}

// The general epilogue's row operands z[r] and w[r], loaded when the row index
// is known and before the row's sum, so that their latency overlaps the tile's
// copy and gathers instead of following the sum (the row-block kernels end each
// tile with a block barrier, so a load issued after the sum stalls the block).
// out_row_pre is final_write with those operands already in registers.
template <class T> struct EpiRow {
    T z, w;
};

template <int MODE, class T> __device__ __forceinline__ EpiRow<T> epi_row_load(const Epi<T> &e, int64_t r)
{
    EpiRow<T> o{T(0), T(0)};
    if constexpr (MODE == 0) {
        if (e.z) o.z = e.z[r];
        if (e.w) o.w = e.w[r];
    } else if constexpr (MODE == 4 || MODE == 5) {
        o.w = e.w[r];
    } else if constexpr (MODE == 7) {
        o.z = e.z[r];
    }
    return o;
}

template <int MODE, class T>
__device__ __forceinline__ void out_row_pre(const Epi<T> &e, int64_t r, T t, const EpiRow<T> &pre, T &d0, T &d1)
{
    if constexpr (MODE == 0) {
        if (!is_one(e.alpha)) t *= e.alpha;
        if (e.z) t = fma(e.beta, pre.z, t);
        e.y[r] = t;
        if (e.w) d0 = fma(pre.w, t, d0);
        if (e.want_yy) d1 = fma(t, t, d1);
    } else if constexpr (MODE >= 4) {
        const T v = MODE == 7 ? fma(T(1), pre.z, -t) : t;
        e.y[r] = v;
        if constexpr (MODE == 4 || MODE == 5) d0 = fma(pre.w, v, d0);
        if constexpr (MODE >= 5) d1 = fma(v, v, d1);
    } else {
        out_row<MODE>(e, r, t, d0, d1);
    }
}

// Reduce (d0, d1) over the grid; the last block stores dots and runs the
// scalar update.  Every block must call it.
template <class T, int BLOCK>
__device__ __forceinline__ void finish_dots(T d0, T d1, const Epi<T> &e, T *partials,
                                            unsigned *ticket)
{
    grid_dots_finish<T, BLOCK>(d0, d1, e.dots, e.fin, e.fin_state, partials, ticket);
}

// ------------------------------------------------------------------ cross-tile carries
// A tile whose end falls inside a row (only rows longer than the tile-map
// slack) publishes that row's partial sum; the tile where the row ends looks
// back over the published partials (decoupled look-back).  Waits only point
// to earlier tiles and the grid is launched cooperatively (all blocks
// resident), so every wait is satisfied; each wait is still bounded.  The
// consumer resets the flag it used, so flags are all zero between launches.
__device__ __forceinline__ void flag_publish(int *flag)
{
    __threadfence();
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(flag), "r"(1) : "memory");
}

__device__ __forceinline__ bool flag_wait(int *flag, unsigned *err, long long limit_cycles = 2000000000LL)
{
    int v;
    const long long t0 = clock64();
    for (;;) {
        asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v != 0) return true;
        if (clock64() - t0 > limit_cycles) {
            if (err) atomicOr(err, DEVERR_QUEUE_TIMEOUT);
            return false;
        }
        __nanosleep(64);
    }
}

// ------------------------------------------------------------------ CSR vector
// One sub-warp of SW lanes per row; lanes stride over the row, then a
// shuffle reduction inside the sub-warp.  The loop is warp-uniform so every
// lane reaches every shuffle.
template <class T, int SW, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    k_csr_vector(int64_t n, const int *__restrict__ rp, const int *__restrict__ col,
                 const T *__restrict__ val, const T *__restrict__ x, Epi<T> e, T *partials,
                 unsigned *ticket)
{
    if (e.skip && *e.skip) return;
    constexpr int RPW = 32 / SW;
    const int lane = threadIdx.x & 31, sub = lane / SW, sl = lane % SW;
    const int64_t warp = (blockIdx.x * (int64_t)BLOCK + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * BLOCK) >> 5;
    T d0 = T(0), d1 = T(0);
    for (int64_t base = warp * RPW; base < n; base += nwarps * RPW) {
        const int64_t i = base + sub;
        T s = T(0);
        if (i < n) {
            const int lo = rp[i], hi = rp[i + 1];
            for (int k = lo + sl; k < hi; k += SW) s = fma(val[k], __ldg(x + col[k]), s);
        }
#pragma unroll
        for (int o = SW / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, SW);
        if (i < n && sl == 0) final_write(e, i, s, d0, d1);
    }
    if (e.dots) finish_dots<T, BLOCK>(d0, d1, e, partials, ticket);
}

// ------------------------------------------------------------------ merge-path CSR
// The merge of the row-end list (rp[1..n]) with the nonzero indices 0..nnz-1
// is cut into tiles of about TILE items (a row end or a nonzero each).  Tile
// boundaries are precomputed and snapped forward to the next row end when
// that is at most SLACK items away, so only rows longer than SLACK straddle
// tiles.  A persistent block loops over its tiles; thread 0 prefetches the
// next tile's row pointers, column indices and values into the other
// shared-memory stage with 1-D bulk copies (TMA) while the block works on
// the current one, and keeps the tile coordinates one tile ahead so that
// issuing a copy never waits on a global load.
//   walk:     each thread takes an equal share of the tile's merge items and
//             accumulates sequentially (one FMA per nonzero, all x gathers of
//             the share issued together); a row end costs one shared-memory
//             store of the running sum, so divergent row ends stay cheap;
//   finalise: one thread per row adds the partial sums of the threads before
//             the row's owner that carried the same row (fixed order), applies
//             the epilogue and stores y coalesced.
// The row sums live in the stage buffer after the copied data: a tile with
// R row ends and Z nonzeros copies 4R + (4+V)Z bytes, and R + Z <= TILE +
// SLACK leaves V*R bytes free.
template <class T, int BLOCK, int IPT> struct MergeShape {
    static constexpr int TILE = BLOCK * IPT;
    static constexpr int SLACK = TILE / 4;
    static constexpr int STAGE = (int)((4 + sizeof(T)) * (TILE + SLACK) + 256);
    // stages | carry rows | carry values | search results | tile coords (2 stages) | mbarriers
    static constexpr int OFF_CROW = 2 * STAGE;
    static constexpr int OFF_CVAL = OFF_CROW + BLOCK * 4;
    static constexpr int OFF_RL = OFF_CVAL + BLOCK * (int)sizeof(T);
    static constexpr int OFF_COORD = OFF_RL + (BLOCK + 1) * 4 + 12;
    static constexpr int OFF_BAR = OFF_COORD + 32;
    static constexpr int SMEM = OFF_BAR + 16;
    static constexpr int CH = IPT < 8 ? IPT : 8;  // nonzeros whose x gathers are issued together
};

struct TileRanges {
    int ra, rbytes, ca, cbytes, va, vbytes;
};

template <class T>
__device__ __forceinline__ TileRanges merge_ranges(int n, int i0, int j0, int i1, int j1)
{
    constexpr int VA = 16 / (int)sizeof(T);
    TileRanges g;
    g.ra = i0 & ~3;
    const int rend = min(i1 + 2, n + 1);  // rp[i0 .. i1+1] (clamped at rp[n])
    g.rbytes = ((rend - g.ra + 3) & ~3) * 4;
    g.ca = j0 & ~3;
    g.cbytes = j1 > j0 ? ((j1 - g.ca + 3) & ~3) * 4 : 0;
    g.va = j0 & ~(VA - 1);
    g.vbytes = j1 > j0 ? ((j1 - g.va + VA - 1) & ~(VA - 1)) * (int)sizeof(T) : 0;
    return g;
}

// Threads with an empty share of a tile are transparent to carry chains.
constexpr int kNoCarry = -1, kEmpty = -2;

// the thread whose share [t*items/B, (t+1)*items/B) contains item p (32-bit: items*B < 2^31)
template <int BLOCK> __device__ __forceinline__ int owner_of(int p, int items)
{
    int t = (p * BLOCK) / items;
    while (t > 0 && (t * items) / BLOCK > p) --t;
    while (t + 1 < BLOCK && ((t + 1) * items) / BLOCK <= p) ++t;
    return t;
}

template <class T, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK)
    k_csr_merge(int n, const int *__restrict__ rp, const int *__restrict__ col,
                const T *__restrict__ val, const T *__restrict__ x, const int2 *__restrict__ tiles,
                int ntiles, int *carry_row_g, T *carry_val_g, int *flags, T *partials, unsigned *ticket,
                unsigned *err, Epi<T> e)
{
    using S = MergeShape<T, BLOCK, IPT>;
    constexpr int CH = S::CH;
    if (e.skip && *e.skip) return;
    extern __shared__ __align__(16) unsigned char smem[];
    int *s_crow = reinterpret_cast<int *>(smem + S::OFF_CROW);
    T *s_cval = reinterpret_cast<T *>(smem + S::OFF_CVAL);
    int *s_rl = reinterpret_cast<int *>(smem + S::OFF_RL);
    int4 *s_coord = reinterpret_cast<int4 *>(smem + S::OFF_COORD);  // per stage (i0, j0, i1, j1)
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + S::OFF_BAR);
    const int tid = threadIdx.x;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    __syncthreads();

    // thread 0 only: copy tile t (coordinates a, b) into `stage`
    auto issue = [&](int2 a, int2 b, int stage) {
        s_coord[stage] = make_int4(a.x, a.y, b.x, b.y);
        const TileRanges g = merge_ranges<T>(n, a.x, a.y, b.x, b.y);
        unsigned char *base = smem + stage * S::STAGE;
        mbar_arrive_expect_tx(&bar[stage], (uint32_t)(g.rbytes + g.cbytes + g.vbytes));
        bulk_g2s(base, rp + g.ra, (uint32_t)g.rbytes, &bar[stage]);
        if (g.cbytes) {
            bulk_g2s(base + g.rbytes, col + g.ca, (uint32_t)g.cbytes, &bar[stage]);
            bulk_g2s(base + g.rbytes + g.cbytes, val + g.va, (uint32_t)g.vbytes, &bar[stage]);
        }
    };

    T d0 = T(0), d1 = T(0);
    int it = 0;
    bool ok = true;
    bool pending_prefetch = false;
    int2 na = make_int2(0, 0), nb = make_int2(0, 0);  // thread 0: coordinates of the tile after next
    if (tid == 0 && (int)blockIdx.x < ntiles) {
        issue(tiles[blockIdx.x], tiles[blockIdx.x + 1], 0);
        const int t2 = blockIdx.x + gridDim.x;
        if (t2 < ntiles) {
            na = tiles[t2];
            nb = tiles[t2 + 1];
        }
    }
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int stage = it & 1;
        const int tn = t + gridDim.x;
        pending_prefetch = tn < ntiles;
        if (tid == 0 && tn < ntiles) {
            fence_proxy_async();
            issue(na, nb, stage ^ 1);
            const int t3 = tn + gridDim.x;
            if (t3 < ntiles) {  // load the coordinates one tile ahead
                na = tiles[t3];
                nb = tiles[t3 + 1];
            }
        }
        if (!mbar_wait(&bar[stage], (uint32_t)((it >> 1) & 1), err)) {
            ok = false;
            break;
        }
        const int4 co = s_coord[stage];
        const int i0 = co.x, j0 = co.y, i1 = co.z, j1 = co.w;
        const TileRanges g = merge_ranges<T>(n, i0, j0, i1, j1);
        unsigned char *sb = smem + stage * S::STAGE;
        const int *s_rp = reinterpret_cast<const int *>(sb) + (i0 - g.ra);             // rp[i0 + k]
        const int *s_col = reinterpret_cast<const int *>(sb + g.rbytes) + (j0 - g.ca);  // col[j0 + k]
        const T *s_val = reinterpret_cast<const T *>(sb + g.rbytes + g.cbytes) + (j0 - g.va);
        T *s_res = reinterpret_cast<T *>(sb + g.rbytes + g.cbytes + g.vbytes);          // row sums
        const int rows_avail = i1 - i0;
        const int nz_tile = j1 - j0;
        const int items = rows_avail + nz_tile;

        // --- this thread's share [dl0, dl1): one search, the end comes from the next thread
        const int dl0 = (tid * items) / BLOCK, dl1 = ((tid + 1) * items) / BLOCK;
        int rl0;
        {
            int lo = max(0, dl0 - nz_tile), hi = min(dl0, rows_avail);
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (mid + s_rp[mid + 1] - j0 < dl0) lo = mid + 1;
                else hi = mid;
            }
            rl0 = lo;
        }
        s_rl[tid] = rl0;
        if (tid == 0) s_rl[BLOCK] = rows_avail;
        __syncthreads();
        const int rl1 = s_rl[tid + 1];
        const int jstart = j0 + (dl0 - rl0), jend = j0 + (dl1 - rl1);

        // --- walk: one FMA per nonzero; a row end stores the running sum
        int lr = rl0;  // local row
        int re = i0 + lr < n ? s_rp[lr + 1] : INT_MAX;
        T sum = T(0);
        const int nnz_t = jend - jstart;
        for (int c = 0; c < nnz_t; c += CH) {
            T v[CH], xv[CH];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int k = jstart - j0 + c + u;
                if (c + u < nnz_t) {
                    v[u] = s_val[k];
                    xv[u] = __ldg(x + s_col[k]);
                } else {
                    v[u] = T(0);
                    xv[u] = T(0);
                }
            }
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                if (c + u < nnz_t) {
                    const int jj = jstart + c + u;
                    while (jj >= re) {
                        s_res[lr] = sum;
                        sum = T(0);
                        ++lr;
                        re = i0 + lr < n ? s_rp[lr + 1] : INT_MAX;
                    }
                    sum = fma(v[u], xv[u], sum);
                }
            }
        }
        while (lr < rl1) {
            s_res[lr] = sum;
            sum = T(0);
            ++lr;
        }
        int crow = kNoCarry;
        const int r = i0 + lr;
        if (dl0 == dl1) crow = kEmpty;
        else if (r < n && jend > max(jstart, s_rp[lr])) crow = r;
        s_crow[tid] = crow;
        s_cval[tid] = sum;
        __syncthreads();

        // --- finalise the rows that end in this tile, one thread per row
        for (int q = tid; q < rows_avail; q += BLOCK) {
            const int row = i0 + q;
            T v = s_res[q];
            int k = owner_of<BLOCK>(q + s_rp[q + 1] - j0, items) - 1;
            while (k >= 0 && (s_crow[k] == row || s_crow[k] == kEmpty)) {
                if (s_crow[k] == row) v += s_cval[k];
                --k;
            }
            if (q == 0 && k < 0 && s_rp[0] < j0) {  // the row began in an earlier tile
                for (int tp = t - 1; tp >= 0; --tp) {
                    if (!flag_wait(flags + tp, err)) break;
                    v += ldcg(carry_val_g + tp);
                    flags[tp] = 0;
                    const int2 pa = tiles[tp];
                    if (!(pa.x == row && pa.y > s_rp[0])) break;  // tile tp began at or before the row start
                }
            }
            final_write(e, row, v, d0, d1);
        }
        // --- publish the partial of a row that continues into the next tile
        if (tid == BLOCK - 1 && i1 < n && j1 > s_rp[rows_avail]) {
            T cv = T(0);
            for (int k = BLOCK - 1; k >= 0 && (s_crow[k] == i1 || s_crow[k] == kEmpty); --k)
                if (s_crow[k] == i1) cv += s_cval[k];
            carry_row_g[t] = i1;
            carry_val_g[t] = cv;
            flag_publish(flags + t);
        }
        __syncthreads();
    }
    if (!ok && pending_prefetch) {
        // do not leave a bulk copy in flight into this block's shared memory
        mbar_wait(&bar[(it + 1) & 1], (uint32_t)(((it + 1) >> 1) & 1), err, 200000000LL);
    }
    if (e.dots) finish_dots<T, BLOCK>(d0, d1, e, partials, ticket);
}

// Tile map: boundary t sits on merge diagonal d = min(t * tile, n + nnz) at
// (i, j), i = #{r : r + rp[r+1] < d}, j = d - i.  If that splits row i and the
// end of row i is at most `slack` items further, the boundary moves there.
// Boundaries that still split a row are counted in *nsplit.
__global__ void k_merge_tiles(int n, int nnz, const int *__restrict__ rp, int64_t tile, int64_t slack,
                              int ntiles, int2 *tiles, unsigned *nsplit)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    const int64_t d = min((int64_t)t * tile, (int64_t)n + nnz);
    int64_t lo = max((int64_t)0, d - nnz), hi = min(d, (int64_t)n);
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (mid + rp[mid + 1] < d) lo = mid + 1;
        else hi = mid;
    }
    int i = (int)lo, j = (int)(d - lo);
    if (i < n && j > rp[i]) {
        const int64_t dn = (int64_t)(i + 1) + rp[i + 1];
        if (dn - d <= slack) {
            i = i + 1;
            j = rp[i];
        } else {
            atomicAdd(nsplit, 1u);
        }
    }
    tiles[t] = make_int2(i, j);
}

// Cross-lane completion of one warp chunk.  cr[l] / cv[l]: the row lane l
// left open at its granule end and that partial sum (kNoCarry / kEmpty if
// none).  Returns, for a lane that ends a row begun in earlier lanes
// (has_pend, row rstart, own part pend), the row's total: its own part, the
// parts of the earlier lanes of the same row, and the chunk carry (run_row,
// run_val) if the row reaches back to lane 0.  Also forms the new chunk carry:
// the row still open at lane 31 (nrow, -1 if none) and its partial (nval).
// Called by all 32 lanes.  When some chain is long, or the carried row spans
// more than one lane, one segmented scan in lockstep (5 steps, full-warp FP64
// adds) gives both; otherwise the short chains are walked directly and the
// carry is lane 31's own partial.
template <class T>
__device__ __forceinline__ T chunk_combine(bool has_pend, int rstart, T pend, const int *cr, const T *cv, int lane,
                                           int run_row, T run_val, int &nrow, T &nval)
{
    const int key = cr[lane];
    nrow = cr[31] >= 0 ? cr[31] : -1;
    const unsigned in_row = __ballot_sync(0xffffffffu, nrow >= 0 && key == nrow);
    const int len = __clz(~in_row);  // lanes 31 .. 32-len carry row nrow
    const bool longchain = has_pend && lane >= 4 && cr[lane - 1] == rstart && cr[lane - 2] == rstart &&
                           cr[lane - 3] == rstart && cr[lane - 4] == rstart;
    if (!__any_sync(0xffffffffu, longchain) && len <= 1) {
        nval = T(0);
        if (nrow >= 0) nval = cv[31];
        if (!has_pend) return T(0);
        T tot = pend;
        int k = lane - 1;
        while (k >= 0 && (cr[k] == rstart || cr[k] == kEmpty)) {
            if (cr[k] == rstart) tot += cv[k];
            --k;
        }
        if (k < 0 && rstart == run_row) tot += run_val;
        return tot;
    }
    T sv = key >= 0 ? cv[lane] : T(0);
    int hd = (lane == 0 || cr[lane - 1] != key) ? 1 : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {  // segmented inclusive scan by key
        const T vu = __shfl_up_sync(0xffffffffu, sv, d);
        const int hu = __shfl_up_sync(0xffffffffu, hd, d);
        if (lane >= d) {
            if (!hd) sv += vu;
            hd |= hu;
        }
    }
    const T prev = __shfl_up_sync(0xffffffffu, sv, 1);
    const unsigned meq = __match_any_sync(0xffffffffu, key);
    const unsigned prevmask = __shfl_up_sync(0xffffffffu, meq, 1);
    nval = __shfl_sync(0xffffffffu, sv, 31);
    if (nrow < 0) nval = T(0);
    else if (len == 32 && nrow == run_row) nval += run_val;
    if (!has_pend) return T(0);
    T tot = pend;
    if (lane > 0 && cr[lane - 1] == rstart) {
        tot += prev;
        const unsigned below = (1u << lane) - 1u;
        if ((prevmask & below) == below && rstart == run_row) tot += run_val;
    } else if (lane == 0 && rstart == run_row) {
        tot += run_val;
    }
    return tot;
}

// ------------------------------------------------------------------ row-block CSR (regular rows)
// For matrices whose rows have similar lengths: a persistent block takes
// tiles of ROWS consecutive rows; one thread copies the tile's row pointers,
// column indices and values into shared memory with three 1-D bulk copies
// (double-buffered: the next tile is in flight while this one is reduced),
// and each thread then reduces one row sequentially from shared memory, one
// FMA per stored entry — ELL's arithmetic without ELL's padding.  With TPR > 1
// threads per row (longer rows), TPR adjacent lanes take every TPR-th entry of
// the row and a shuffle adds their sums: more gathers in flight per SM when
// shared memory caps the resident tiles.  `cap` is
// the largest number of nonzeros in any tile (measured on the host), so the
// copies always fit; a tile above it (never, for an unmodified matrix) sets
// DEVERR_BOUNDS and is skipped.
template <class T, int ROWS> struct RowsShape {
    static constexpr int RP_BYTES = (ROWS + 8) * 4;  // rp[r0 - 3 .. r1 + 3], 16-byte rounded
    static __host__ __device__ int col_bytes(int cap) { return ((cap + 8) * 4 + 15) & ~15; }
    static __host__ __device__ int val_bytes(int cap) { return ((cap + 8) * (int)sizeof(T) + 15) & ~15; }
    static __host__ __device__ int stage(int cap) { return RP_BYTES + col_bytes(cap) + val_bytes(cap); }
    // stages | tile coordinates (2 x int4) | mbarriers (2)
    static __host__ __device__ int smem(int cap, int stages) { return stages * stage(cap) + 32 + 16; }
};

template <class T, int ROWS, int STAGES, int MODE, int TPR>
__global__ void __launch_bounds__(ROWS * TPR)
    k_csr_rows(int n, const int *__restrict__ rp, const int *__restrict__ col, const T *__restrict__ val,
               const T *__restrict__ x, int ntiles, int cap, T *partials, unsigned *ticket, unsigned *err, Epi<T> e)
{
    using S = RowsShape<T, ROWS>;
    constexpr int VA = 16 / (int)sizeof(T);
    constexpr int CH = 8;
    static_assert(STAGES == 1 || STAGES == 2, "one or two stages");
    static_assert(TPR == 1 || TPR == 2 || TPR == 4, "1, 2 or 4 threads per row");
    if (e.skip && *e.skip) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int stage_bytes = S::stage(cap);
    int4 *s_coord = reinterpret_cast<int4 *>(smem + STAGES * stage_bytes);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + STAGES * stage_bytes + 32);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int k = 0; k < STAGES; ++k) mbar_init(&bar[k], 1);
        fence_barrier_init();
    }
    __syncthreads();

    // thread 0 only: copy the tile with rows [r0, r1) and nonzeros [j0, j1) into `stage`
    auto issue = [&](int r0, int r1, int j0, int j1, int stage) {
        unsigned char *base = smem + stage * stage_bytes;
        const int ra = r0 & ~3;
        const int rbytes = ((r1 + 1 - ra + 3) & ~3) * 4;
        int ca = j0 & ~3, cbytes = ((j1 - ca + 3) & ~3) * 4;
        int va = j0 & ~(VA - 1), vbytes = ((j1 - va + VA - 1) & ~(VA - 1)) * (int)sizeof(T);
        if (j1 - j0 > cap) {  // cannot happen for the matrix the cap was measured on
            atomicOr(err, DEVERR_BOUNDS);
            j1 = j0;
        }
        if (j1 == j0) cbytes = vbytes = 0;
        s_coord[stage] = make_int4(r0, j0, r1, j1);
        mbar_arrive_expect_tx(&bar[stage], (uint32_t)(rbytes + cbytes + vbytes));
        bulk_g2s(base, rp + ra, (uint32_t)rbytes, &bar[stage]);
        if (cbytes) {
            bulk_g2s(base + S::RP_BYTES, col + ca, (uint32_t)cbytes, &bar[stage]);
            bulk_g2s(base + S::RP_BYTES + S::col_bytes(cap), val + va, (uint32_t)vbytes, &bar[stage]);
        }
    };

    T d0 = T(0), d1 = T(0);
    int it = 0;
    bool ok = true, pending_prefetch = false;
    // thread 0: the next tile to copy (tile index, nonzero range), loaded one copy ahead
    int nt = blockIdx.x, nj0 = 0, nj1 = 0;
    auto load_next = [&]() {
        if (nt < ntiles) {
            nj0 = rp[nt * ROWS];
            nj1 = rp[min(n, nt * ROWS + ROWS)];
        }
    };
    auto issue_next = [&](int stage) {
        if (nt < ntiles) issue(nt * ROWS, min(n, nt * ROWS + ROWS), nj0, nj1, stage);
        nt += gridDim.x;
        load_next();
    };
    if (tid == 0) {
        load_next();
        if (STAGES == 2) issue_next(0);
    }
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int stage = STAGES == 2 ? (it & 1) : 0;
        if (STAGES == 2) {
            pending_prefetch = t + (int)gridDim.x < ntiles;
            if (tid == 0) {
                fence_proxy_async();
                issue_next(stage ^ 1);  // the tile after this one
            }
        } else if (tid == 0) {
            fence_proxy_async();
            issue_next(0);  // this tile
        }
        const int q = tid / TPR, sub = tid % TPR;  // this thread's row of the tile; its lane within the row
        const int rq = t * ROWS + q;
        const EpiRow<T> pre = rq < n && sub == 0 ? epi_row_load<MODE>(e, rq) : EpiRow<T>{T(0), T(0)};
        const uint32_t parity = STAGES == 2 ? (uint32_t)((it >> 1) & 1) : (uint32_t)(it & 1);
        bool waited = mbar_wait(&bar[stage], parity, err);
        if constexpr (TPR > 1) waited = __all_sync(0xffffffffu, waited);  // the shuffle below needs whole warps
        if (!waited) {
            ok = false;
            break;
        }
        const int4 co = s_coord[stage];
        const int r0 = co.x, j0 = co.y, r1 = co.z, j1 = co.w;
        const unsigned char *sb = smem + stage * stage_bytes;
        const int *s_rp = reinterpret_cast<const int *>(sb) + (r0 - (r0 & ~3));
        const int *s_col = reinterpret_cast<const int *>(sb + S::RP_BYTES) + (j0 - (j0 & ~3));
        const T *s_val = reinterpret_cast<const T *>(sb + S::RP_BYTES + S::col_bytes(cap)) + (j0 - (j0 & ~(VA - 1)));
        const bool live = r0 + q < r1;
        T sum = T(0);
        if (live) {
            const int a0 = s_rp[q] - j0;
            const int len = (j1 > j0 ? s_rp[q + 1] - j0 : a0) - a0;
            // this lane's entries: a0 + sub + TPR*u for u < mine.  Every lane of a row
            // steps through cnt = ceil(len / TPR) slots, a lane's slots past its own
            // entries adding 0 * 0: the FMA sequence is then the same in every lane of
            // the row (with a per-lane count, rows whose length is not a multiple of
            // TPR ran both tail branches in one warp, one FP64 instruction more per row
            // pair on the 27-point stencil)
            const int cnt = TPR == 1 ? len : (len + TPR - 1) / TPR;
            const int mine = TPR == 1 ? len : (len - sub + TPR - 1) / TPR;
            const int *pc = s_col + a0 + sub;
            const T *pv = s_val + a0 + sub;
            int a = 0;
            for (; a + CH <= cnt; a += CH) {  // full chunks: CH gathers in flight, then CH FMAs
                T v[CH], xv[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    const bool real = TPR == 1 || a + u < mine;
                    v[u] = real ? pv[(a + u) * TPR] : T(0);
                    xv[u] = real ? __ldg(x + pc[(a + u) * TPR]) : T(0);
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) sum = fma(v[u], xv[u], sum);
            }
            const int rem = cnt - a;  // 0 .. CH-1: gathers issued together, FMAs only for the row's slots
            if (rem > 0) {
                T v[CH - 1], xv[CH - 1];
#pragma unroll
                for (int u = 0; u < CH - 1; ++u) {
                    const bool real = u < rem && (TPR == 1 || a + u < mine);
                    v[u] = real ? pv[(a + u) * TPR] : T(0);
                    xv[u] = real ? __ldg(x + pc[(a + u) * TPR]) : T(0);
                }
                if (rem & 4) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) sum = fma(v[u], xv[u], sum);
                    v[0] = v[4]; v[1] = v[5]; v[2] = v[6];
                    xv[0] = xv[4]; xv[1] = xv[5]; xv[2] = xv[6];
                }
                if (rem & 2) {
                    sum = fma(v[0], xv[0], sum);
                    sum = fma(v[1], xv[1], sum);
                    v[0] = v[2];
                    xv[0] = xv[2];
                }
                if (rem & 1) sum = fma(v[0], xv[0], sum);
            }
        }
        if constexpr (TPR > 1) {  // lanes of a row are adjacent and in one warp; every lane takes part
#pragma unroll
            for (int o = TPR / 2; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o, TPR);
        }
        if (live && sub == 0) out_row_pre<MODE>(e, r0 + q, sum, pre, d0, d1);
        __syncthreads();  // the stage is refilled by a later copy
    }
    if (!ok && pending_prefetch) {
        // do not leave a bulk copy in flight into this block's shared memory
        mbar_wait(&bar[(it + 1) & 1], (uint32_t)(((it + 1) >> 1) & 1), err, 200000000LL);
    }
    if constexpr (MODE == 0 || MODE >= 4)
        if (e.dots) finish_dots<T, ROWS * TPR>(d0, d1, e, partials, ticket);
}

// ------------------------------------------------------------------ row-block COO (regular rows)
// The COO counterpart of k_csr_rows: tiles of ROWS consecutive rows, whose
// entries [tiles[t], tiles[t+1]) are bulk-copied (row indices, columns,
// values) into shared memory, double-buffered.  The block then marks where
// the staged row indices change, which gives every row its range inside the
// tile, and each thread reduces one row with one FMA per entry.
template <class T, int ROWS> struct CooRowsShape {
    static __host__ __device__ int idx_bytes(int cap) { return ((cap + 8) * 4 + 15) & ~15; }
    static __host__ __device__ int val_bytes(int cap) { return ((cap + 8) * (int)sizeof(T) + 15) & ~15; }
    static __host__ __device__ int stage(int cap) { return 2 * idx_bytes(cap) + val_bytes(cap); }
    static __host__ __device__ int smem(int cap) { return 2 * stage(cap) + 32 + 16; }
};

template <class T, int ROWS, int MODE>
__global__ void __launch_bounds__(ROWS)
    k_coo_rows(int n, const int *__restrict__ crow, const int *__restrict__ ccol, const T *__restrict__ cval,
               const T *__restrict__ x, const int *__restrict__ tiles, int ntiles, int cap, T *partials,
               unsigned *ticket, unsigned *err, Epi<T> e)
{
    using S = CooRowsShape<T, ROWS>;
    constexpr int VA = 16 / (int)sizeof(T);
    constexpr int CH = 8;
    if (e.skip && *e.skip) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_first[ROWS], s_end[ROWS];
    const int stage_bytes = S::stage(cap);
    int4 *s_coord = reinterpret_cast<int4 *>(smem + 2 * stage_bytes);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * stage_bytes + 32);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    __syncthreads();

    // thread 0 only: copy tile t's entries [e0, e1) into `stage`
    auto issue = [&](int t, int e0, int e1, int stage) {
        unsigned char *base = smem + stage * stage_bytes;
        if (e1 - e0 > cap) {  // cannot happen for the matrix the cap was measured on
            atomicOr(err, DEVERR_BOUNDS);
            e1 = e0;
        }
        const int ia = e0 & ~3, ibytes = e1 > e0 ? ((e1 - ia + 3) & ~3) * 4 : 0;
        const int va = e0 & ~(VA - 1), vbytes = e1 > e0 ? ((e1 - va + VA - 1) & ~(VA - 1)) * (int)sizeof(T) : 0;
        s_coord[stage] = make_int4(t * ROWS, e0, min(n, t * ROWS + ROWS), e1);
        mbar_arrive_expect_tx(&bar[stage], (uint32_t)(2 * ibytes + vbytes));
        if (ibytes) {
            bulk_g2s(base, crow + ia, (uint32_t)ibytes, &bar[stage]);
            bulk_g2s(base + S::idx_bytes(cap), ccol + ia, (uint32_t)ibytes, &bar[stage]);
            bulk_g2s(base + 2 * S::idx_bytes(cap), cval + va, (uint32_t)vbytes, &bar[stage]);
        }
    };

    T d0 = T(0), d1 = T(0);
    int it = 0;
    bool ok = true, pending_prefetch = false;
    int ne0 = 0, ne1 = 0;  // thread 0: entry range of the tile after next
    if (tid == 0 && (int)blockIdx.x < ntiles) {
        issue(blockIdx.x, tiles[blockIdx.x], tiles[blockIdx.x + 1], 0);
        const int t2 = (int)blockIdx.x + (int)gridDim.x;
        if (t2 < ntiles) {
            ne0 = tiles[t2];
            ne1 = tiles[t2 + 1];
        }
    }
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int stage = it & 1;
        const int tn = t + gridDim.x;
        pending_prefetch = tn < ntiles;
        if (tid == 0 && tn < ntiles) {
            fence_proxy_async();
            issue(tn, ne0, ne1, stage ^ 1);
            const int t3 = tn + gridDim.x;
            if (t3 < ntiles) {
                ne0 = tiles[t3];
                ne1 = tiles[t3 + 1];
            }
        }
        s_first[tid] = 0;
        s_end[tid] = 0;
        const int rq = t * ROWS + tid;  // this thread's row of the tile
        const EpiRow<T> pre = rq < n ? epi_row_load<MODE>(e, rq) : EpiRow<T>{T(0), T(0)};
        if (!mbar_wait(&bar[stage], (uint32_t)((it >> 1) & 1), err)) {
            ok = false;
            break;
        }
        const int4 co = s_coord[stage];
        const int r0 = co.x, e0 = co.y, r1 = co.z, e1 = co.w;
        const unsigned char *sb = smem + stage * stage_bytes;
        const int *s_row = reinterpret_cast<const int *>(sb) + (e0 - (e0 & ~3));
        const int *s_col = reinterpret_cast<const int *>(sb + S::idx_bytes(cap)) + (e0 - (e0 & ~3));
        const T *s_val = reinterpret_cast<const T *>(sb + 2 * S::idx_bytes(cap)) + (e0 - (e0 & ~(VA - 1)));
        const int cnt = e1 - e0;
        __syncthreads();  // s_first / s_end cleared
        for (int k = tid; k < cnt; k += ROWS) {  // where the row index changes: row starts and ends
            const int rk = s_row[k];
            if (k == 0 || s_row[k - 1] != rk) s_first[rk - r0] = k;
            if (k == cnt - 1 || s_row[k + 1] != rk) s_end[rk - r0] = k + 1;
        }
        __syncthreads();
        const int q = tid;
        if (r0 + q < r1) {
            int a = s_first[q];
            const int b = s_end[q];
            T sum = T(0);
            for (; a + CH <= b; a += CH) {
                T v[CH], xv[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    v[u] = s_val[a + u];
                    xv[u] = __ldg(x + s_col[a + u]);
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) sum = fma(v[u], xv[u], sum);
            }
            const int rem = b - a;
            if (rem > 0) {
                T v[CH - 1], xv[CH - 1];
#pragma unroll
                for (int u = 0; u < CH - 1; ++u) {
                    v[u] = u < rem ? s_val[a + u] : T(0);
                    xv[u] = u < rem ? __ldg(x + s_col[a + u]) : T(0);
                }
                if (rem & 4) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) sum = fma(v[u], xv[u], sum);
                    v[0] = v[4]; v[1] = v[5]; v[2] = v[6];
                    xv[0] = xv[4]; xv[1] = xv[5]; xv[2] = xv[6];
                }
                if (rem & 2) {
                    sum = fma(v[0], xv[0], sum);
                    sum = fma(v[1], xv[1], sum);
                    v[0] = v[2];
                    xv[0] = xv[2];
                }
                if (rem & 1) sum = fma(v[0], xv[0], sum);
            }
            out_row_pre<MODE>(e, r0 + q, sum, pre, d0, d1);
        }
        __syncthreads();  // the stage and the row marks are reused
    }
    if (!ok && pending_prefetch) mbar_wait(&bar[(it + 1) & 1], (uint32_t)(((it + 1) >> 1) & 1), err, 200000000LL);
    if constexpr (MODE == 0 || MODE >= 4)
        if (e.dots) finish_dots<T, ROWS>(d0, d1, e, partials, ticket);
}

// tiles[t] = first COO entry of row t * rows (entries are row-sorted), t = 0..ntiles
__global__ void k_coo_rowtiles(int n, int64_t nnz, const int *__restrict__ crow, int rows, int ntiles, int *tiles,
                               int *maxcnt)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    const int r = min(n, t * rows);
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (crow[mid] < r) lo = mid + 1;
        else hi = mid;
    }
    tiles[t] = (int)lo;
    if (t > 0) {  // entries of tile t-1: lower_bound of its first row, recomputed
        const int rp = min(n, (t - 1) * rows);
        int64_t a = 0, b = nnz;
        while (a < b) {
            const int64_t mid = (a + b) >> 1;
            if (crow[mid] < rp) a = mid + 1;
            else b = mid;
        }
        atomicMax(maxcnt, (int)(lo - a));
    }
}

// the largest number of nonzeros in a tile of `rows` consecutive rows
__global__ void k_tile_max_nnz(int n, const int *__restrict__ rp, int rows, int ntiles, int *out)
{
    int m = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x)
        m = max(m, rp[min(n, (t + 1) * rows)] - rp[t * rows]);
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ------------------------------------------------------------------ nnz-split CSR (warp-independent)
// Every lane of a persistent warp takes a granule of IPT consecutive nonzeros
// (loads fully independent of any search: coalesced across the warp) and
// finds its first row through a row hint (hint[g] = row holding nonzero
// g*IPT).  It accumulates sequentially, one FMA per nonzero, and writes y for
// every row that ends inside its granule.  A row that began in an earlier
// lane of the same chunk is completed from those lanes' partial sums (a short
// chain in shared memory); a row running past the chunk is carried to the
// warp's next chunk in registers.  Each warp owns one contiguous range of
// chunks, so only the row straddling a range boundary crosses warps: the
// warp publishes that partial when it finishes and completes its own first
// row last, looking back at the previous warps (cooperative launch).  No
// block-wide barrier is needed until the final dot reduction.
//   Row ownership: row r ends in the lane whose granule [a, b) has
//   a < rp[r+1] <= b (rows with rp[r+1] == 0 belong to granule 0).
template <class T, int IPT, int MODE>
__global__ void __launch_bounds__(256)
    k_csr_split(int n, int nnz, const int *__restrict__ rp, const int *__restrict__ col,
                const T *__restrict__ val, const T *__restrict__ x, const int *__restrict__ hint, int nchunks,
                int *carry_row_w, T *carry_val_w, int *flags, T *partials, unsigned *ticket, unsigned *err,
                Epi<T> e)
{
    constexpr int CH = IPT == 8 ? 4 : 8;  // gathers issued together (4: fewer registers, 8-wide granules)
    constexpr int NW = 256 / 32;
    constexpr int CHUNK = 32 * IPT, PADDED = CHUNK + 32;  // element k sits at k + k / IPT
    if (e.skip && *e.skip) return;
    __shared__ int s_cr[NW][32];
    __shared__ T s_cv[NW][32];
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *sc = reinterpret_cast<int *>(smem_dyn) + wib * PADDED;
    T *sv = reinterpret_cast<T *>(smem_dyn + (size_t)NW * PADDED * 4) + wib * PADDED;
    const int W = gridDim.x * NW;
    const int w = blockIdx.x * NW + wib;
    const int c_begin = (int)(((int64_t)nchunks * w) / W), c_end = (int)(((int64_t)nchunks * (w + 1)) / W);
    T d0 = T(0), d1 = T(0);

    // the range's first row, if it began before the range, is completed last
    const int64_t range_a = (int64_t)c_begin * 32 * IPT;
    int first_row = -1;
    bool range_inside = false;
    if (c_begin < c_end && range_a < nnz) {
        first_row = hint[(int64_t)c_begin * 32];
        range_inside = rp[first_row] < range_a;
    }
    T first_val = T(0);
    bool first_ready = false;   // the first row ended in this range (value in first_val, lane 0)
    int run_row = -1;           // row carried from the previous chunk (warp-uniform)
    T run_val = T(0);

    for (int c = c_begin; c < c_end; ++c) {
        const int64_t g = (int64_t)c * 32 + lane;
        const int64_t a = g * IPT;
        const int b = (int)min(a + IPT, (int64_t)nnz);
        const bool active = a < nnz;
        {  // coalesced copy of the chunk's columns and values into padded shared memory
            const int64_t a0 = (int64_t)c * CHUNK;
            const int cc = (int)min((int64_t)CHUNK, (int64_t)nnz - a0);
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                const int kq = lane + 32 * q;
                if (kq < cc) {
                    sc[kq + kq / IPT] = col[a0 + kq];
                    sv[kq + kq / IPT] = val[a0 + kq];
                }
            }
            __syncwarp();
        }
        int r = active ? hint[g] : n;
        int re = r < n ? rp[r + 1] : INT_MAX;
        const bool pend_possible = active && rp[r] < a;
        T sum = T(0), pend = T(0);
        bool first = true, has_pend = false;
        const int rstart = r;
#define SPX_SPLIT_EMIT(row_, s_)                       \
    do {                                               \
        if (first && pend_possible) {                  \
            pend = (s_);                               \
            has_pend = true;                           \
        } else {                                       \
            out_row<MODE>(e, (row_), (s_), d0, d1);    \
        }                                              \
        first = false;                                 \
    } while (0)
        if (a == 0 && active)  // rows before the first nonzero have no entries
            for (int q = 0; q < r; ++q) out_row<MODE>(e, q, T(0), d0, d1);
        if (active) {
            const int cnt = b - (int)a;
#pragma unroll
            for (int kk = 0; kk < IPT; kk += CH) {
                T v[CH], xv[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    if (kk + u < cnt) {
                        v[u] = sv[lane * (IPT + 1) + kk + u];
                        xv[u] = __ldg(x + sc[lane * (IPT + 1) + kk + u]);
                    } else {
                        v[u] = T(0);
                        xv[u] = T(0);
                    }
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    const int j = (int)a + kk + u;
                    if (kk + u < cnt && j >= re) {  // divergent, but free of FP64 work
                        do {
                            SPX_SPLIT_EMIT(r, sum);
                            sum = T(0);
                            ++r;
                            re = r < n ? rp[r + 1] : INT_MAX;
                        } while (j >= re);
                    }
                    sum = fma(v[u], xv[u], sum);  // unused slots hold zeros: uniform across the warp
                }
            }
            while (r < n && re <= b) {  // rows ending exactly at b (and empty rows there)
                SPX_SPLIT_EMIT(r, sum);
                sum = T(0);
                ++r;
                re = r < n ? rp[r + 1] : INT_MAX;
            }
        }
        int cr = kEmpty;
        if (active) cr = (r < n && b > max((int)a, rp[r])) ? r : kNoCarry;
        s_cr[wib][lane] = cr;
        s_cv[wib][lane] = sum;
        __syncwarp();
        // complete a row that began in earlier lanes (and maybe earlier chunks);
        // carry the row still open at lane 31 to the next chunk
        int nrow;
        T nval;
        const T tot = chunk_combine<T>(has_pend, rstart, pend, s_cr[wib], s_cv[wib], lane, run_row, run_val, nrow,
                                       nval);
        if (has_pend) {
            if (range_inside && rstart == first_row) {
                first_val = tot;  // finished last, after the look-back
                first_ready = true;
            } else {
                out_row<MODE>(e, rstart, tot, d0, d1);
            }
        }
        run_row = nrow;
        run_val = nval;
        // the lane that finished the deferred first row passes it to lane 0
        const unsigned fm = __ballot_sync(0xffffffffu, first_ready);
        if (fm) {
            const int src = __ffs(fm) - 1;
            first_val = __shfl_sync(0xffffffffu, first_val, src);
            first_ready = true;
        }
        __syncwarp();
    }
    // publish the partial of the row that continues into the next warp's range
    if (lane == 0 && run_row >= 0) {
        carry_row_w[w] = run_row;
        carry_val_w[w] = run_val;
        flag_publish(flags + w);
    }
    // then complete the range's first row from the previous ranges' partials
    if (lane == 0 && range_inside && first_ready) {
        T tot = first_val;
        const int rs = rp[first_row];
        for (int wp = w - 1; wp >= 0; --wp) {
            const int pb = (int)(((int64_t)nchunks * wp) / W), pe = (int)(((int64_t)nchunks * (wp + 1)) / W);
            if (pb >= pe) continue;  // empty range
            if (!flag_wait(flags + wp, err)) break;
            tot += ldcg(carry_val_w + wp);
            flags[wp] = 0;
            if (!(rs < (int64_t)pb * 32 * IPT)) break;  // range wp began at or before the row start
        }
        out_row<MODE>(e, first_row, tot, d0, d1);
    }
    if constexpr (MODE == 0 || MODE >= 4)
        if (e.dots) finish_dots<T, 256>(d0, d1, e, partials, ticket);
#undef SPX_SPLIT_EMIT
}

// ------------------------------------------------------------------ tiled nnz-split CSR
// The lane-granule decomposition of k_csr_split on a copy of the nonzeros
// laid out for it once per matrix.  In a chunk of 32 granules of IPT
// consecutive nonzeros, slot u of lane l is stored at
//     (u / VEC) * 32 VEC + l VEC + u % VEC,  VEC = elements per 16 bytes,
// so one 16-byte load per lane reads VEC slots of all 32 lanes coalesced, and
// the chunk goes straight to registers (no shared-memory staging, whose
// stores and loads share the L1 data path with the random gathers of x).
// Row boundaries come from a per-granule descriptor instead of row pointers:
// trow[g] = the row holding the granule's first nonzero (bit 31 set when an
// empty row lies between two rows of the granule), tmask[g] bit u = a row
// starts at slot u.  So the only dependent loads in a granule are the
// gathers.  Empty rows are listed once per matrix and written (t = 0) by all
// threads at the start; flagged granules step over them through the row
// pointers.  Lanes, chunks and warp ranges are combined as in k_csr_split.
// (Storing a tile transposed with per-tile row descriptors follows the CSR5
// format of Liu and Vinter, ICS 2015; written from that description.)
template <class T, int IPT, int MODE>
__global__ void __launch_bounds__(256)
    k_csr_tiled(int n, int nnz, const int *__restrict__ rp, const int *__restrict__ tcol,
                const T *__restrict__ tval, const int *__restrict__ trow, const unsigned *__restrict__ tmask,
                const int *__restrict__ empty, int nempty, const T *__restrict__ x, int nchunks, int *carry_row_w,
                T *carry_val_w, int *flags, T *partials, unsigned *ticket, unsigned *err, Epi<T> e)
{
    constexpr int CH = 8;                    // gathers issued together
    constexpr int VC = 4;                    // column slots per 16-byte load
    constexpr int VV = 16 / (int)sizeof(T);  // value slots per 16-byte load
    constexpr int NW = 256 / 32;
    constexpr int CHUNK = 32 * IPT;
    static_assert(IPT % CH == 0 && CH % VC == 0 && CH % VV == 0 && IPT <= 32, "tiled CSR shape");
    if (e.skip && *e.skip) return;
    __shared__ int s_cr[NW][32];
    __shared__ T s_cv[NW][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int W = gridDim.x * NW;
    const int w = blockIdx.x * NW + wib;
    T d0 = T(0), d1 = T(0);
    for (int q = blockIdx.x * 256 + threadIdx.x; q < nempty; q += gridDim.x * 256)
        out_row<MODE>(e, empty[q], T(0), d0, d1);
    const int c_begin = (int)(((int64_t)nchunks * w) / W), c_end = (int)(((int64_t)nchunks * (w + 1)) / W);

    // the range's first row, if it began before the range, is completed last
    const int64_t range_a = (int64_t)c_begin * CHUNK;
    int first_row = -1;
    bool range_inside = false;
    if (c_begin < c_end && range_a < nnz) {
        first_row = trow[(int64_t)c_begin * 32] & 0x7fffffff;
        range_inside = (tmask[(int64_t)c_begin * 32] & 1u) == 0u;
    }
    T first_val = T(0);
    bool first_ready = false;
    int run_row = -1;
    T run_val = T(0);

    for (int c = c_begin; c < c_end; ++c) {
        const int64_t g = (int64_t)c * 32 + lane;
        const int64_t a = g * IPT;
        const int cnt = (int)max((int64_t)0, min((int64_t)IPT, (int64_t)nnz - a));
        const bool active = cnt > 0;
        const int rd = trow[g];
        const unsigned m = tmask[g];
        const bool ends_b = a + IPT >= nnz || (tmask[g + 1] & 1u) != 0u;  // the last row ends with the granule
        const bool slow = rd < 0;
        int r = rd & 0x7fffffff;
        const int rstart = r;
        const bool pend_possible = active && (m & 1u) == 0u;
        T sum = T(0), pend = T(0);
        bool first = true, has_pend = false;
        const int *cp = tcol + (int64_t)c * CHUNK + lane * VC;
        const T *vp = tval + (int64_t)c * CHUNK + lane * VV;
#define SPX_TILED_EMIT(row_, s_)                       \
    do {                                               \
        if (first && pend_possible) {                  \
            pend = (s_);                               \
            has_pend = true;                           \
        } else {                                       \
            out_row<MODE>(e, (row_), (s_), d0, d1);    \
        }                                              \
        first = false;                                 \
    } while (0)
#pragma unroll
        for (int kk = 0; kk < IPT; kk += CH) {
            int cc[CH];
            T v[CH], xv[CH];
#pragma unroll
            for (int q = 0; q < CH / VC; ++q) {
                const int4 t4 = __ldcs(reinterpret_cast<const int4 *>(cp + (kk / VC + q) * 32 * VC));
                cc[4 * q + 0] = t4.x;
                cc[4 * q + 1] = t4.y;
                cc[4 * q + 2] = t4.z;
                cc[4 * q + 3] = t4.w;
            }
#pragma unroll
            for (int q = 0; q < CH / VV; ++q) {
                if constexpr (sizeof(T) == 8) {
                    const double2 t2 = __ldcs(reinterpret_cast<const double2 *>(vp + (kk / VV + q) * 32 * VV));
                    v[2 * q + 0] = t2.x;
                    v[2 * q + 1] = t2.y;
                } else {
                    const float4 t4 = __ldcs(reinterpret_cast<const float4 *>(vp + (kk / VV + q) * 32 * VV));
                    v[4 * q + 0] = t4.x;
                    v[4 * q + 1] = t4.y;
                    v[4 * q + 2] = t4.z;
                    v[4 * q + 3] = t4.w;
                }
            }
#pragma unroll
            for (int u = 0; u < CH; ++u) xv[u] = kk + u < cnt ? __ldg(x + cc[u]) : T(0);
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int sl = kk + u;
                if (sl > 0 && sl < cnt && ((m >> sl) & 1u)) {  // a row starts here: the previous one is complete
                    SPX_TILED_EMIT(r, sum);
                    sum = T(0);
                    if (slow) {  // step over empty rows (written at the start)
                        ++r;
                        while (rp[r + 1] == rp[r]) ++r;
                    } else {
                        ++r;
                    }
                }
                if (sl < cnt) sum = fma(v[u], xv[u], sum);
            }
        }
        int cr = kEmpty;
        if (active) {
            if (ends_b) {
                SPX_TILED_EMIT(r, sum);
                sum = T(0);
                cr = kNoCarry;
            } else {
                cr = r;
            }
        }
#undef SPX_TILED_EMIT
        s_cr[wib][lane] = cr;
        s_cv[wib][lane] = sum;
        __syncwarp();
        int nrow;
        T nval;
        const T tot = chunk_combine<T>(has_pend, rstart, pend, s_cr[wib], s_cv[wib], lane, run_row, run_val, nrow,
                                       nval);
        if (has_pend) {
            if (range_inside && rstart == first_row) {
                first_val = tot;
                first_ready = true;
            } else {
                out_row<MODE>(e, rstart, tot, d0, d1);
            }
        }
        run_row = nrow;
        run_val = nval;
        const unsigned fm = __ballot_sync(0xffffffffu, first_ready);
        if (fm) {
            const int src = __ffs(fm) - 1;
            first_val = __shfl_sync(0xffffffffu, first_val, src);
            first_ready = true;
        }
        __syncwarp();
    }
    if (lane == 0 && run_row >= 0) {
        carry_row_w[w] = run_row;
        carry_val_w[w] = run_val;
        flag_publish(flags + w);
    }
    if (lane == 0 && range_inside && first_ready) {
        T tot = first_val;
        const int rs = rp[first_row];
        for (int wp = w - 1; wp >= 0; --wp) {
            const int pb = (int)(((int64_t)nchunks * wp) / W), pe = (int)(((int64_t)nchunks * (wp + 1)) / W);
            if (pb >= pe) continue;
            if (!flag_wait(flags + wp, err)) break;
            tot += ldcg(carry_val_w + wp);
            flags[wp] = 0;
            if (!(rs < (int64_t)pb * CHUNK)) break;
        }
        out_row<MODE>(e, first_row, tot, d0, d1);
    }
    if constexpr (MODE == 0 || MODE >= 4)
        if (e.dots) finish_dots<T, 256>(d0, d1, e, partials, ticket);
}

// Tiled copy of the nonzeros: source entry k (thread k) goes to its slot in
// the transposed chunk layout; the padded slots past nnz hold column 0 and
// value 0 (never used: the kernel predicates on the granule's count).
template <class T, int VEC>
__global__ void k_tile_transpose(int64_t nnz, int64_t total, int ipt, const T *__restrict__ src, T *__restrict__ dst)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= total) return;
    const int64_t chunk = 32LL * ipt;
    const int64_t c = k / chunk;
    const int wi = (int)(k - c * chunk);
    const int l = wi / ipt, u = wi - l * ipt;
    dst[c * chunk + (int64_t)(u / VEC) * 32 * VEC + l * VEC + u % VEC] = k < nnz ? src[k] : T(0);
}

// Granule descriptors, step 1: trow[g] = the row holding nonzero g * ipt
// (the first row r with rp[r+1] > g * ipt, so never an empty row); tmask
// cleared.  Granules past nnz get row 0.
__global__ void k_tile_rows(int n, int64_t nnz, const int *__restrict__ rp, int ipt, int64_t ngran, int *trow,
                            unsigned *tmask)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g > ngran) return;
    tmask[g] = 0u;
    if (g == ngran) return;
    const int64_t a = g * ipt;
    int r = 0;
    if (a < nnz) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((int64_t)rp[mid + 1] > a) hi = mid;
            else lo = mid + 1;
        }
        r = lo;
    }
    trow[g] = r;
}

// Step 2, one thread per row: a non-empty row sets the bit of its first slot;
// an empty row that falls strictly inside a granule flags that granule.
__global__ void k_tile_marks(int n, int64_t nnz, const int *__restrict__ rp, int ipt, int *trow, unsigned *tmask)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int p = rp[r];
    const int64_t g = p / ipt;
    const int u = p - (int)(g * ipt);
    if (rp[r + 1] > p) atomicOr(tmask + g, 1u << u);
    else if (u != 0 && p < nnz) atomicOr(reinterpret_cast<unsigned *>(trow + g), 0x80000000u);
}

// Empty rows in increasing order (one block: deterministic, so the kernels'
// dot products sum them in a fixed order).  *count receives their number.
__global__ void __launch_bounds__(1024) k_empty_rows(int n, const int *__restrict__ rp, int *out, int *count)
{
    __shared__ int s[1024];
    const int t = threadIdx.x;
    const int64_t r0 = (int64_t)n * t / 1024, r1 = (int64_t)n * (t + 1) / 1024;
    int c = 0;
    for (int64_t r = r0; r < r1; ++r) c += rp[r + 1] == rp[r];
    s[t] = c;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan
        const int v = t >= o ? s[t - o] : 0;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    int pos = s[t] - c;
    if (out)
        for (int64_t r = r0; r < r1; ++r)
            if (rp[r + 1] == rp[r]) out[pos++] = (int)r;
    if (t == 1023) *count = s[1023];
}

// ------------------------------------------------------------------ nnz-split COO (warp-independent)
// The COO counterpart of k_csr_split: lane granules of IPT consecutive
// entries, the row of every entry read from the row array.  A lane ends row r
// at its last entry when the next entry's row differs; rows without entries
// between two entries are written (store mode) by the lane that sees the
// jump.  Carries between lanes, chunks and warp ranges as in k_csr_split.
// Add mode (the COO part of HYB) adds alpha * sum into y and writes no gaps.
template <class T, int IPT, int MODE>
__global__ void __launch_bounds__(256)
    k_coo_split(int n, int nnz, const int *__restrict__ crow, const int *__restrict__ ccol,
                const T *__restrict__ cval, const T *__restrict__ x, int nchunks, int *carry_row_w,
                T *carry_val_w, int *flags, T *partials, unsigned *ticket, unsigned *err, Epi<T> e)
{
    constexpr bool add_mode = MODE == 2 || MODE == 3;  // y += ..., no rows without entries written
    constexpr int CH = IPT == 8 ? 4 : 8;  // gathers issued together (4: fewer registers, 8-wide granules)
    constexpr int NW = 256 / 32;
    constexpr int CHUNK = 32 * IPT, PADDED = CHUNK + 32;  // element k sits at k + k / IPT
    if (e.skip && *e.skip) return;
    __shared__ int s_cr[NW][32];
    __shared__ T s_cv[NW][32];
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *sc = reinterpret_cast<int *>(smem_dyn) + wib * PADDED;
    int *sr = reinterpret_cast<int *>(smem_dyn) + (NW + wib) * PADDED;
    T *sv = reinterpret_cast<T *>(smem_dyn + (size_t)2 * NW * PADDED * 4) + wib * PADDED;
    const int W = gridDim.x * NW;
    const int w = blockIdx.x * NW + wib;
    const int c_begin = (int)(((int64_t)nchunks * w) / W), c_end = (int)(((int64_t)nchunks * (w + 1)) / W);
    T d0 = T(0), d1 = T(0);
#define SPX_COO_OUT(row_, s_) out_row<MODE>(e, (row_), (s_), d0, d1)

    const int64_t range_a = (int64_t)c_begin * 32 * IPT;
    int first_row = -1;
    bool range_inside = false;
    if (c_begin < c_end && range_a < nnz) {
        first_row = crow[range_a];
        range_inside = range_a > 0 && crow[range_a - 1] == first_row;
    }
    T first_val = T(0);
    bool first_ready = false;
    int run_row = -1;
    T run_val = T(0);

    for (int c = c_begin; c < c_end; ++c) {
        const int64_t g = (int64_t)c * 32 + lane;
        const int64_t a = g * IPT;
        const int b = (int)min(a + IPT, (int64_t)nnz);
        const bool active = a < nnz;
        {  // coalesced copy of the chunk's rows, columns and values into padded shared memory
            const int64_t a0 = (int64_t)c * CHUNK;
            const int cc = (int)min((int64_t)CHUNK, (int64_t)nnz - a0);
#pragma unroll
            for (int q = 0; q < IPT; ++q) {
                const int kq = lane + 32 * q;
                if (kq < cc) {
                    sr[kq + kq / IPT] = crow[a0 + kq];
                    sc[kq + kq / IPT] = ccol[a0 + kq];
                    sv[kq + kq / IPT] = cval[a0 + kq];
                }
            }
            __syncwarp();
        }
        int r = active ? sr[lane * (IPT + 1)] : n;
        const bool pend_possible = active && a > 0 && crow[a - 1] == r;
        const int rstart = r;
        T sum = T(0), pend = T(0);
        bool first = true, has_pend = false;
#define SPX_COO_EMIT(row_, s_)                                                     \
    do {                                                                           \
        if (first && pend_possible) {                                              \
            pend = (s_);                                                           \
            has_pend = true;                                                       \
        } else {                                                                   \
            SPX_COO_OUT(row_, s_);                                                 \
        }                                                                          \
        first = false;                                                             \
    } while (0)
        if (a == 0 && active && !add_mode)
            for (int q = 0; q < r; ++q) out_row<MODE>(e, q, T(0), d0, d1);  // rows before the first entry
        int cr = kEmpty;
        if (active) {
            const int cnt = b - (int)a;
#pragma unroll
            for (int kk = 0; kk < IPT; kk += CH) {
                T v[CH], xv[CH];
                int rr[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    if (kk + u < cnt) {
                        v[u] = sv[lane * (IPT + 1) + kk + u];
                        xv[u] = __ldg(x + sc[lane * (IPT + 1) + kk + u]);
                        rr[u] = sr[lane * (IPT + 1) + kk + u];
                    } else {
                        v[u] = T(0);
                        xv[u] = T(0);
                        rr[u] = r;
                    }
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    if (kk + u < cnt && rr[u] != r) {  // divergent, but free of FP64 work
                        SPX_COO_EMIT(r, sum);
                        if (!add_mode)
                            for (int q = r + 1; q < rr[u]; ++q) out_row<MODE>(e, q, T(0), d0, d1);
                        r = rr[u];
                        sum = T(0);
                    }
                    sum = fma(v[u], xv[u], sum);  // unused slots hold zeros: uniform across the warp
                }
            }
            const int nr = b < nnz ? crow[b] : n;
            if (nr == r) {
                cr = r;
            } else {
                SPX_COO_EMIT(r, sum);
                if (!add_mode)
                    for (int q = r + 1; q < nr; ++q) out_row<MODE>(e, q, T(0), d0, d1);
                sum = T(0);
                cr = kNoCarry;
            }
        }
        s_cr[wib][lane] = cr;
        s_cv[wib][lane] = sum;
        __syncwarp();
        int nrow;
        T nval;
        const T tot = chunk_combine<T>(has_pend, rstart, pend, s_cr[wib], s_cv[wib], lane, run_row, run_val, nrow,
                                       nval);
        if (has_pend) {
            if (range_inside && rstart == first_row) {
                first_val = tot;
                first_ready = true;
            } else {
                SPX_COO_OUT(rstart, tot);
            }
        }
        run_row = nrow;
        run_val = nval;
        const unsigned fm = __ballot_sync(0xffffffffu, first_ready);
        if (fm) {
            const int src = __ffs(fm) - 1;
            first_val = __shfl_sync(0xffffffffu, first_val, src);
            first_ready = true;
        }
        __syncwarp();
#undef SPX_COO_EMIT
    }
    if (lane == 0 && run_row >= 0) {
        carry_row_w[w] = run_row;
        carry_val_w[w] = run_val;
        flag_publish(flags + w);
    }
    if (lane == 0 && range_inside && first_ready) {
        T tot = first_val;
        for (int wp = w - 1; wp >= 0; --wp) {
            const int pb = (int)(((int64_t)nchunks * wp) / W), pe = (int)(((int64_t)nchunks * (wp + 1)) / W);
            if (pb >= pe) continue;
            if (!flag_wait(flags + wp, err)) break;
            tot += ldcg(carry_val_w + wp);
            flags[wp] = 0;
            const int64_t ps = (int64_t)pb * 32 * IPT;
            if (!(ps > 0 && crow[ps - 1] == first_row)) break;  // range wp began at the row start
        }
        SPX_COO_OUT(first_row, tot);
    }
    if constexpr (MODE == 0 || MODE >= 4)
        if (e.dots) finish_dots<T, 256>(d0, d1, e, partials, ticket);
#undef SPX_COO_OUT
}

// ------------------------------------------------------------------ tiled nnz-split COO
// k_coo_split on tile-transposed copies of the row, column and value arrays
// (the layout of k_csr_tiled): a lane's granule arrives by coalesced 16-byte
// loads straight into registers.  Row boundaries come from the row indices
// themselves, as the COO format defines them.  The rows on either side of a
// granule (entries a-1 and b) come from the neighbouring lanes by shuffles
// once the granule is summed (reading them from memory would cost a sector
// per granule edge: a quarter more DRAM traffic at 16 entries per lane), so
// the decision whether the granule's first row continues one begun earlier is
// taken after the loop.  Rows without entries are written by the lane that
// sees the jump; carries as in k_coo_split.
template <class T, int IPT, int MODE>
__global__ void __launch_bounds__(256, 4)
    k_coo_tiled(int n, int nnz, const int *__restrict__ crow, const int *__restrict__ trowi,
                const int *__restrict__ tcol, const T *__restrict__ tval, const T *__restrict__ x, int nchunks,
                int *carry_row_w, T *carry_val_w, int *flags, T *partials, unsigned *ticket, unsigned *err, Epi<T> e)
{
    constexpr bool add_mode = MODE == 2 || MODE == 3;
    constexpr int CH = sizeof(T) == 8 ? 4 : 8;
    constexpr int VC = 4, VV = 16 / (int)sizeof(T);
    constexpr int NW = 256 / 32;
    constexpr int CHUNK = 32 * IPT;
    static_assert(IPT % CH == 0 && CH % VC == 0 && CH % VV == 0 && IPT <= 32, "tiled COO shape");
    if (e.skip && *e.skip) return;
    __shared__ int s_cr[NW][32];
    __shared__ T s_cv[NW][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int W = gridDim.x * NW;
    const int w = blockIdx.x * NW + wib;
    const int c_begin = (int)(((int64_t)nchunks * w) / W), c_end = (int)(((int64_t)nchunks * (w + 1)) / W);
    T d0 = T(0), d1 = T(0);

    const int64_t range_a = (int64_t)c_begin * CHUNK;
    int first_row = -1;
    bool range_inside = false;
    int prev_last = -1;  // row of the entry before the current chunk (warp-uniform)
    if (c_begin < c_end && range_a < nnz) {
        first_row = crow[range_a];
        prev_last = range_a > 0 ? crow[range_a - 1] : -1;
        range_inside = prev_last == first_row;
    }
    T first_val = T(0);
    bool first_ready = false;
    int run_row = -1;
    T run_val = T(0);

    for (int c = c_begin; c < c_end; ++c) {
        const int64_t g = (int64_t)c * 32 + lane;
        const int64_t a = g * IPT;
        const int cnt = (int)max((int64_t)0, min((int64_t)IPT, (int64_t)nnz - a));
        const bool active = cnt > 0;
        const int b = (int)(a + cnt);
        // the row after the chunk's last entry (lane 31's neighbour), one load per chunk
        const int after_chunk = lane == 31 && active && b < nnz ? crow[b] : n;
        const int *rq = trowi + (int64_t)c * CHUNK + lane * VC;
        const int *cp = tcol + (int64_t)c * CHUNK + lane * VC;
        const T *vp = tval + (int64_t)c * CHUNK + lane * VV;
        int r = active ? __ldcs(rq) : n;
        const int r0 = r;
        T sum = T(0), head = T(0);
        bool have_head = false;
        if (active) {
#pragma unroll
            for (int kk = 0; kk < IPT; kk += CH) {
                int rr[CH], cc[CH];
                T v[CH], xv[CH];
#pragma unroll
                for (int q = 0; q < CH / VC; ++q) {
                    const int4 r4 = __ldcs(reinterpret_cast<const int4 *>(rq + (kk / VC + q) * 32 * VC));
                    const int4 c4 = __ldcs(reinterpret_cast<const int4 *>(cp + (kk / VC + q) * 32 * VC));
                    rr[4 * q + 0] = r4.x;
                    rr[4 * q + 1] = r4.y;
                    rr[4 * q + 2] = r4.z;
                    rr[4 * q + 3] = r4.w;
                    cc[4 * q + 0] = c4.x;
                    cc[4 * q + 1] = c4.y;
                    cc[4 * q + 2] = c4.z;
                    cc[4 * q + 3] = c4.w;
                }
#pragma unroll
                for (int q = 0; q < CH / VV; ++q) {
                    if constexpr (sizeof(T) == 8) {
                        const double2 t2 = __ldcs(reinterpret_cast<const double2 *>(vp + (kk / VV + q) * 32 * VV));
                        v[2 * q + 0] = t2.x;
                        v[2 * q + 1] = t2.y;
                    } else {
                        const float4 t4 = __ldcs(reinterpret_cast<const float4 *>(vp + (kk / VV + q) * 32 * VV));
                        v[4 * q + 0] = t4.x;
                        v[4 * q + 1] = t4.y;
                        v[4 * q + 2] = t4.z;
                        v[4 * q + 3] = t4.w;
                    }
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) xv[u] = kk + u < cnt ? __ldg(x + cc[u]) : T(0);
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    if (kk + u < cnt && rr[u] != r) {  // a segment ends: the first one waits for the neighbours
                        if (!have_head) {
                            head = sum;
                            have_head = true;
                        } else {
                            out_row<MODE>(e, r, sum, d0, d1);
                        }
                        if (!add_mode)
                            for (int q = r + 1; q < rr[u]; ++q) out_row<MODE>(e, q, T(0), d0, d1);
                        r = rr[u];
                        sum = T(0);
                    }
                    if (kk + u < cnt) sum = fma(v[u], xv[u], sum);
                }
            }
        }
        // the neighbours' rows: entry a-1 ends lane l-1's granule, entry b starts lane l+1's
        int prev = __shfl_up_sync(0xffffffffu, r, 1);
        if (lane == 0) prev = prev_last;
        int nr = __shfl_down_sync(0xffffffffu, r0, 1);
        if (lane == 31 || b >= nnz) nr = lane == 31 ? after_chunk : n;
        prev_last = __shfl_sync(0xffffffffu, r, 31);
        const bool pend_possible = active && prev == r0;
        const int rstart = r0;
        T pend = T(0);
        bool has_pend = false;
        int cr = kEmpty;
        if (active) {
            if (!add_mode && prev + 1 < r0)  // rows without entries between the previous granule and this one
                for (int q = prev + 1; q < r0; ++q) out_row<MODE>(e, q, T(0), d0, d1);
            if (have_head) {  // the first segment ended inside the granule
                if (pend_possible) {
                    pend = head;
                    has_pend = true;
                } else {
                    out_row<MODE>(e, r0, head, d0, d1);
                }
            }
            if (nr == r) {  // the last segment continues into the next granule
                cr = r;
            } else {
                if (!have_head && pend_possible) {
                    pend = sum;
                    has_pend = true;
                } else {
                    out_row<MODE>(e, r, sum, d0, d1);
                }
                if (!add_mode && b >= nnz)  // rows without entries after the last entry
                    for (int q = r + 1; q < n; ++q) out_row<MODE>(e, q, T(0), d0, d1);
                sum = T(0);
                cr = kNoCarry;
            }
        }
        s_cr[wib][lane] = cr;
        s_cv[wib][lane] = sum;
        __syncwarp();
        int nrow;
        T nval;
        const T tot = chunk_combine<T>(has_pend, rstart, pend, s_cr[wib], s_cv[wib], lane, run_row, run_val, nrow,
                                       nval);
        if (has_pend) {
            if (range_inside && rstart == first_row) {
                first_val = tot;
                first_ready = true;
            } else {
                out_row<MODE>(e, rstart, tot, d0, d1);
            }
        }
        run_row = nrow;
        run_val = nval;
        const unsigned fm = __ballot_sync(0xffffffffu, first_ready);
        if (fm) {
            const int src = __ffs(fm) - 1;
            first_val = __shfl_sync(0xffffffffu, first_val, src);
            first_ready = true;
        }
        __syncwarp();
    }
    if (lane == 0 && run_row >= 0) {
        carry_row_w[w] = run_row;
        carry_val_w[w] = run_val;
        flag_publish(flags + w);
    }
    if (lane == 0 && range_inside && first_ready) {
        T tot = first_val;
        for (int wp = w - 1; wp >= 0; --wp) {
            const int pb = (int)(((int64_t)nchunks * wp) / W), pe = (int)(((int64_t)nchunks * (wp + 1)) / W);
            if (pb >= pe) continue;
            if (!flag_wait(flags + wp, err)) break;
            tot += ldcg(carry_val_w + wp);
            flags[wp] = 0;
            const int64_t ps = (int64_t)pb * CHUNK;
            if (!(ps > 0 && crow[ps - 1] == first_row)) break;  // range wp began at the row start
        }
        out_row<MODE>(e, first_row, tot, d0, d1);
    }
    if constexpr (MODE == 0 || MODE >= 4)
        if (e.dots) finish_dots<T, 256>(d0, d1, e, partials, ticket);
}

// hint[g] = the row holding nonzero g*ipt: first r with rp[r+1] > g*ipt
__global__ void k_row_hint(int n, int nnz, const int *__restrict__ rp, int ipt, int ng, int *hint)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int64_t j = (int64_t)g * ipt;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (rp[mid + 1] > j) hi = mid;
        else lo = mid + 1;
    }
    hint[g] = lo;
}

// ------------------------------------------------------------------ ELL
// Column-major ELL [width][ld]: thread g handles rows g*R .. g*R+R-1 and
// reads R consecutive values (16 B for R = 16 / sizeof(T)) per slab, fully
// coalesced across the warp.  Padding slots (col = -1) are skipped.
template <class T, int R> struct Vec;
template <> struct Vec<double, 1> { using V = double; using I = int; };
template <> struct Vec<double, 2> { using V = double2; using I = int2; };
template <> struct Vec<float, 1> { using V = float; using I = int; };
template <> struct Vec<float, 2> { using V = float2; using I = int2; };
template <> struct Vec<float, 4> { using V = float4; using I = int4; };

template <class T, int R, int BLOCK, int MODE>
__global__ void __launch_bounds__(BLOCK)
    k_ell(int64_t n, int64_t ld, int w, const int *__restrict__ ecol, const T *__restrict__ eval,
          const T *__restrict__ x, Epi<T> e, T *partials, unsigned *ticket)
{
    if (e.skip && *e.skip) return;
    using VV = typename Vec<T, R>::V;
    using VI = typename Vec<T, R>::I;
    constexpr int U = 4;  // slabs whose loads are issued together
    T d0 = T(0), d1 = T(0);
    const int64_t ngroups = (n + R - 1) / R;
    for (int64_t g = blockIdx.x * (int64_t)BLOCK + threadIdx.x; g < ngroups;
         g += (int64_t)gridDim.x * BLOCK) {
        const int64_t i = g * R;
        T s[R];
#pragma unroll
        for (int q = 0; q < R; ++q) s[q] = T(0);
        int j = 0;
        for (; j + U <= w; j += U) {
            VI c[U];
            VV v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t o = (int64_t)(j + u) * ld + i;
                c[u] = __ldg(reinterpret_cast<const VI *>(ecol + o));
                v[u] = __ldg(reinterpret_cast<const VV *>(eval + o));
            }
            T xg[U][R];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int *cc = reinterpret_cast<const int *>(&c[u]);
#pragma unroll
                for (int q = 0; q < R; ++q) xg[u][q] = cc[q] >= 0 ? __ldg(x + cc[q]) : T(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const T *vv = reinterpret_cast<const T *>(&v[u]);
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    if constexpr (sizeof(T) == 8) {  // FP64 pipe is scarce: skip padding slots
                        if (reinterpret_cast<const int *>(&c[u])[q] >= 0) s[q] = fma(vv[q], xg[u][q], s[q]);
                    } else {
                        s[q] = fma(vv[q], xg[u][q], s[q]);  // padding multiplies 0 * 0
                    }
                }
            }
        }
        for (; j < w; ++j) {
            const int64_t o = (int64_t)j * ld + i;
            const VI c = __ldg(reinterpret_cast<const VI *>(ecol + o));
            const VV v = __ldg(reinterpret_cast<const VV *>(eval + o));
            const int *cc = reinterpret_cast<const int *>(&c);
            const T *vv = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int q = 0; q < R; ++q)
                if (cc[q] >= 0) s[q] = fma(vv[q], __ldg(x + cc[q]), s[q]);
        }
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (i + q < n) out_row<MODE>(e, i + q, s[q], d0, d1);
    }
    if constexpr (MODE == 0 || MODE >= 4)
        if (e.dots) finish_dots<T, BLOCK>(d0, d1, e, partials, ticket);
}

// ------------------------------------------------------------------ COO segmented reduction
// Tiles of about TILE nonzeros (row-sorted COO, boundaries snapped forward to
// the next row start when it is at most SLACK entries away) are staged by
// bulk copies.  walk: each thread reduces an equal share of the tile's
// entries sequentially; when the row index changes, the finished sum goes
// into the shared-memory value slot of the row's last entry (a slot only
// this thread reads, already consumed).  finalise: one thread per row end
// adds the carries of the threads before the owner (fixed order) and stores
// y; rows without entries get alpha*0 + beta*z.  Add mode (the COO part of
// HYB) adds into y instead.  Rows that straddle tiles use the look-back.
template <class T, int BLOCK, int IPT> struct CooShape {
    static constexpr int TILE = BLOCK * IPT;
    static constexpr int SLACK = TILE / 4;
    static constexpr int STAGE = (int)((8 + sizeof(T)) * (TILE + SLACK) + 128);
    // stages | carry rows | carry values | tile coords (2 stages) | mbarriers
    static constexpr int OFF_CROW = 2 * STAGE;
    static constexpr int OFF_CVAL = OFF_CROW + BLOCK * 4;
    static constexpr int OFF_COORD = OFF_CVAL + BLOCK * (int)sizeof(T);
    static constexpr int OFF_BAR = OFF_COORD + 32;
    static constexpr int SMEM = OFF_BAR + 16;
    static constexpr int CH = IPT < 8 ? IPT : 8;
};

template <class T>
__device__ __forceinline__ TileRanges coo_ranges(int64_t k0, int64_t k1)
{
    constexpr int VA = 16 / (int)sizeof(T);
    TileRanges g;
    g.ra = (int)(k0 & ~3LL);
    g.rbytes = (int)(((k1 - g.ra + 3) & ~3LL) * 4);
    g.ca = g.ra;
    g.cbytes = g.rbytes;
    g.va = (int)(k0 & ~(int64_t)(VA - 1));
    g.vbytes = (int)(((k1 - g.va + VA - 1) & ~(int64_t)(VA - 1)) * sizeof(T));
    return g;
}

template <class T, int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK)
    k_coo(int64_t n, int64_t nnz, const int *__restrict__ crow, const int *__restrict__ ccol,
          const T *__restrict__ cval, const T *__restrict__ x, const int *__restrict__ tiles, int ntiles,
          int *carry_row_g, T *carry_val_g, int *flags, T *partials, unsigned *ticket, unsigned *err, Epi<T> e,
          int add_mode)
{
    using S = CooShape<T, BLOCK, IPT>;
    constexpr int CH = S::CH;
    if (e.skip && *e.skip) return;
    extern __shared__ __align__(16) unsigned char smem[];
    int *s_crow = reinterpret_cast<int *>(smem + S::OFF_CROW);
    T *s_cval = reinterpret_cast<T *>(smem + S::OFF_CVAL);
    int4 *s_coord = reinterpret_cast<int4 *>(smem + S::OFF_COORD);  // (k0, k1, row before, row after)
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + S::OFF_BAR);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    __syncthreads();

    auto coords = [&](int t) -> int4 {  // thread 0, one tile ahead of its use
        const int k0 = tiles[t], k1 = tiles[t + 1];
        return make_int4(k0, k1, k0 > 0 ? __ldg(crow + k0 - 1) : -1, k1 < nnz ? __ldg(crow + k1) : (int)n);
    };
    auto issue = [&](int4 c, int stage) {
        s_coord[stage] = c;
        const int64_t k0 = c.x, k1 = c.y;
        unsigned char *base = smem + stage * S::STAGE;
        if (k1 <= k0) {  // empty tile: complete the phase with no bytes
            mbar_arrive_expect_tx(&bar[stage], 0u);
            return;
        }
        const TileRanges g = coo_ranges<T>(k0, k1);
        mbar_arrive_expect_tx(&bar[stage], (uint32_t)(2 * g.rbytes + g.vbytes));
        bulk_g2s(base, crow + g.ra, (uint32_t)g.rbytes, &bar[stage]);
        bulk_g2s(base + g.rbytes, ccol + g.ca, (uint32_t)g.cbytes, &bar[stage]);
        bulk_g2s(base + 2 * g.rbytes, cval + g.va, (uint32_t)g.vbytes, &bar[stage]);
    };

    T d0 = T(0), d1 = T(0);
    int it = 0;
    bool ok = true, pending_prefetch = false;
    int4 nc = make_int4(0, 0, 0, 0);  // thread 0: coordinates of the tile after next
    if (tid == 0 && (int)blockIdx.x < ntiles) {
        issue(coords(blockIdx.x), 0);
        if ((int)(blockIdx.x + gridDim.x) < ntiles) nc = coords(blockIdx.x + gridDim.x);
    }
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int stage = it & 1;
        const int tn = t + gridDim.x;
        pending_prefetch = tn < ntiles;
        if (tid == 0 && tn < ntiles) {
            fence_proxy_async();
            issue(nc, stage ^ 1);
            if (tn + (int)gridDim.x < ntiles) nc = coords(tn + gridDim.x);
        }
        if (!mbar_wait(&bar[stage], (uint32_t)((it >> 1) & 1), err)) {
            ok = false;
            break;
        }
        const int4 co = s_coord[stage];
        const int64_t kt0 = co.x, kt1 = co.y;
        const int row_before = co.z, row_after = co.w;
        const TileRanges g = coo_ranges<T>(kt0, max(kt1, kt0 + 1));
        unsigned char *sb = smem + stage * S::STAGE;
        const int *s_row = reinterpret_cast<const int *>(sb) + (kt0 - g.ra);
        const int *s_col = reinterpret_cast<const int *>(sb + g.rbytes) + (kt0 - g.ca);
        T *s_val = reinterpret_cast<T *>(sb + 2 * g.rbytes) + (kt0 - g.va);
        const int tile_n = (int)(kt1 - kt0);
        const int l0 = (tid * tile_n) / BLOCK, l1 = ((tid + 1) * tile_n) / BLOCK;
        auto row_at = [&](int64_t k) -> int {  // row of entry k in [kt0, kt1]
            return k < kt1 ? s_row[k - kt0] : row_after;
        };
        // --- walk
        T sum = T(0);
        int crow_out = kEmpty;
        if (l0 < l1) {
            int r = s_row[l0];
            const int cnt = l1 - l0;
            for (int c = 0; c < cnt; c += CH) {
                T v[CH], xv[CH];
                int rr[CH];
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    const int k = l0 + c + u;
                    if (c + u < cnt) {
                        v[u] = s_val[k];
                        xv[u] = __ldg(x + s_col[k]);
                        rr[u] = s_row[k];
                    } else {
                        v[u] = T(0);
                        xv[u] = T(0);
                        rr[u] = r;
                    }
                }
#pragma unroll
                for (int u = 0; u < CH; ++u) {
                    if (c + u < cnt) {
                        if (rr[u] != r) {  // entry l0+c+u-1 ended row r
                            s_val[l0 + c + u - 1] = sum;
                            r = rr[u];
                            sum = T(0);
                        }
                        sum = fma(v[u], xv[u], sum);
                    }
                }
            }
            if (row_at(kt0 + l1) == r) {
                crow_out = r;
            } else {
                s_val[l1 - 1] = sum;
                sum = T(0);
                crow_out = kNoCarry;
            }
        }
        s_crow[tid] = crow_out;
        s_cval[tid] = sum;
        __syncthreads();
        // --- finalise: one thread per entry that ends a row in this tile
        if (tid == 0 && kt0 == 0 && tile_n > 0 && !add_mode)
            for (int q = 0; q < s_row[0]; ++q) final_write(e, q, T(0), d0, d1);  // rows before the first entry
        for (int q = tid; q < tile_n; q += BLOCK) {
            const int row = s_row[q];
            const int next = q + 1 < tile_n ? s_row[q + 1] : row_after;
            if (next == row) continue;  // not the row's last entry
            T v = s_val[q];
            int k = owner_of<BLOCK>(q, tile_n) - 1;
            while (k >= 0 && (s_crow[k] == row || s_crow[k] == kEmpty)) {
                if (s_crow[k] == row) v += s_cval[k];
                --k;
            }
            if (k < 0 && row_before == row) {  // the row began in an earlier tile
                for (int tp = t - 1; tp >= 0; --tp) {
                    if (!flag_wait(flags + tp, err)) break;
                    v += ldcg(carry_val_g + tp);
                    flags[tp] = 0;
                    const int64_t ps = tiles[tp];
                    if (!(ps > 0 && __ldg(crow + ps) == row && __ldg(crow + ps - 1) == row)) break;
                }
            }
            if (add_mode) {
                e.y[row] += e.alpha * v;
            } else {
                final_write(e, row, v, d0, d1);
                for (int gq = row + 1; gq < next; ++gq) final_write(e, gq, T(0), d0, d1);  // rows without entries
            }
        }
        if (tid == BLOCK - 1 && kt1 < nnz && kt1 > kt0 && s_row[tile_n - 1] == row_after) {
            const int cr = s_row[tile_n - 1];
            T cv = T(0);
            for (int k = BLOCK - 1; k >= 0 && (s_crow[k] == cr || s_crow[k] == kEmpty); --k)
                if (s_crow[k] == cr) cv += s_cval[k];
            carry_row_g[t] = cr;
            carry_val_g[t] = cv;
            flag_publish(flags + t);
        }
        __syncthreads();
    }
    if (!ok && pending_prefetch)
        mbar_wait(&bar[(it + 1) & 1], (uint32_t)(((it + 1) >> 1) & 1), err, 200000000LL);
    if (e.dots && !add_mode) finish_dots<T, BLOCK>(d0, d1, e, partials, ticket);
}

// COO tile map: boundary t at entry k = min(t * tile, nnz), moved forward to
// the start of the next row when that is at most `slack` entries away.
__global__ void k_coo_tiles(int64_t nnz, const int *__restrict__ crow, int64_t tile, int64_t slack, int ntiles,
                            int *tiles, unsigned *nsplit)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    int64_t k = min((int64_t)t * tile, nnz);
    if (k > 0 && k < nnz && crow[k - 1] == crow[k]) {
        const int r = crow[k];
        const int64_t hi = min(k + slack, nnz);
        if (hi < nnz && crow[hi] == r) {
            atomicAdd(nsplit, 1u);  // the row runs on past the slack: keep the split
        } else {  // first q in [k, hi] with q == nnz or crow[q] != r
            int64_t lo = k, h = hi;
            while (lo < h) {
                const int64_t mid = (lo + h) >> 1;
                if (crow[mid] == r) lo = mid + 1;
                else h = mid;
            }
            k = lo;
        }
    }
    tiles[t] = (int)k;
}

// ------------------------------------------------------------------ whole-vector epilogue
// y = beta * z (alpha * A x with no stored entries), used for empty matrices.
template <class T, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    k_scale_only(int64_t n, Epi<T> e, T *partials, unsigned *ticket)
{
    if (e.skip && *e.skip) return;
    T d0 = T(0), d1 = T(0);
    for (int64_t i = blockIdx.x * (int64_t)BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * BLOCK)
        final_write(e, i, T(0), d0, d1);
    if (e.dots) finish_dots<T, BLOCK>(d0, d1, e, partials, ticket);
}

// dots over an already stored y (HYB needs them after both parts are added)
template <class T, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    k_dots_of_y(int64_t n, Epi<T> e, T *partials, unsigned *ticket)
{
    if (e.skip && *e.skip) return;
    T d0 = T(0), d1 = T(0);
    for (int64_t i = blockIdx.x * (int64_t)BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * BLOCK) {
        const T v = e.y[i];
        if (e.w) d0 = fma(e.w[i], v, d0);
        if (e.want_yy) d1 = fma(v, v, d1);
    }
    finish_dots<T, BLOCK>(d0, d1, e, partials, ticket);
}

// ------------------------------------------------------------------ host side
namespace {

constexpr int kVecBlock = 256;
constexpr int kEllBlock = 256;
constexpr int kMergeBlock = 256;
constexpr int kCooBlock = 256;

template <class K> int grid_for(spx_ctx *ctx, K kernel, int block, int smem, int64_t work_blocks)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t g = (int64_t)per_sm * ctx->grid_sms;
    if (g > work_blocks) g = work_blocks;
    return (int)(g < 1 ? 1 : g);
}

std::mutex g_smem_mu;
std::map<std::pair<const void *, int>, int> g_smem_granted;  // (kernel, device) -> dynamic bytes

}  // namespace

int smem_optin(const void *kernel, int bytes, int *granted)
{
    int dev = 0;
    SPX_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_smem_mu);
    const auto key = std::make_pair(kernel, dev);
    auto it = g_smem_granted.find(key);
    if (it == g_smem_granted.end() || (bytes >= 0 && bytes > it->second)) {
        int want = bytes;
        if (want < 0) {
            cudaFuncAttributes fa;
            int optin = 0;
            SPX_CUDA(cudaFuncGetAttributes(&fa, kernel));
            SPX_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
            want = optin - (int)fa.sharedSizeBytes;
        }
        const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(max dynamic shared memory)");
        it = g_smem_granted.insert_or_assign(key, want).first;
    }
    if (granted) *granted = it->second;
    return SPX_OK;
}

namespace {

template <class K> int set_smem(K kernel, int bytes)
{
    return smem_optin(reinterpret_cast<const void *>(kernel), bytes);
}

// Scratch (carries, look-back flags, partials, ticket) sized for the largest
// grid / tile count seen.  Flags start at zero and are left at zero by every
// launch (each consumer resets the flag it used).
int ensure_scratch(spx_ctx *ctx, spx_matrix *A, int64_t ntiles, int64_t grid, size_t vbytes)
{
    const size_t need_c = (size_t)(ntiles + 1);
    if (A->carry_row.bytes < need_c * 4) {
        dbuf_free(ctx, A->carry_row);
        dbuf_free(ctx, A->carry_val);
        dbuf_free(ctx, A->flags);
        SPX_TRY(dbuf_alloc(ctx, A->carry_row, need_c * 4));
        SPX_TRY(dbuf_alloc(ctx, A->carry_val, need_c * 8));
        SPX_TRY(dbuf_alloc(ctx, A->flags, need_c * 4));
        SPX_CUDA(cudaMemsetAsync(A->flags.p, 0, need_c * 4, ctx->stream));
    }
    const size_t need_p = (size_t)(2 * grid + 2) * 8;
    if (A->partials.bytes < need_p) {
        dbuf_free(ctx, A->partials);
        SPX_TRY(dbuf_alloc(ctx, A->partials, need_p));
    }
    if (!A->ticket.p) {
        SPX_TRY(dbuf_alloc(ctx, A->ticket, 64));
        SPX_CUDA(cudaMemsetAsync(A->ticket.p, 0, 64, ctx->stream));
    }
    (void)vbytes;
    return SPX_OK;
}

// Launch, cooperatively when blocks may wait on one another (look-back).
template <class... KArgs, class... Args>
int launch_k(void (*kern)(KArgs...), int grid, int block, int smem, cudaStream_t st, bool coop, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = coop ? at : nullptr;
    cfg.numAttrs = coop ? 1 : 0;
    SPX_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
    return SPX_OK;
}

int ensure_coo_tiles(spx_ctx *ctx, spx_matrix *A, int64_t tile_items, int64_t slack)
{
    if (A->coo_tiles.p && A->coo_tiles_items == tile_items) return SPX_OK;
    const int64_t ntiles = ceil_div(A->coo_nnz, tile_items);
    if (ntiles + 1 > INT_MAX) return fail(SPX_ERR_TOO_LARGE, "too many COO tiles");
    dbuf_free(ctx, A->coo_tiles);
    SPX_TRY(dbuf_alloc(ctx, A->coo_tiles, (size_t)(ntiles + 1) * 4 + 16));
    unsigned *cnt = reinterpret_cast<unsigned *>(A->coo_tiles.as<int>() + ntiles + 1);
    SPX_CUDA(cudaMemsetAsync(cnt, 0, 4, ctx->stream));
    k_coo_tiles<<<(int)ceil_div(ntiles + 1, 256), 256, 0, ctx->stream>>>(
        A->coo_nnz, A->coo_row.as<int>(), tile_items, slack, (int)ntiles, A->coo_tiles.as<int>(), cnt);
    SPX_CUDA(cudaGetLastError());
    unsigned h = 0;
    SPX_CUDA(cudaMemcpyAsync(&h, cnt, 4, cudaMemcpyDeviceToHost, ctx->stream));
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    A->coo_tiles_items = tile_items;
    A->coo_ntiles = ntiles;
    A->coo_nsplit = h;
    return SPX_OK;
}

template <class T, int IPT>
int launch_merge(spx_ctx *ctx, spx_matrix *A, const T *val, const T *x, const Epi<T> &e)
{
    using S = MergeShape<T, kMergeBlock, IPT>;
    auto kern = k_csr_merge<T, kMergeBlock, IPT>;
    SPX_TRY(ensure_merge_tiles(ctx, A, S::TILE, S::SLACK));
    SPX_TRY(set_smem(kern, S::SMEM));
    const int grid = grid_for(ctx, kern, kMergeBlock, S::SMEM, A->ntiles);
    SPX_TRY(ensure_scratch(ctx, A, A->ntiles, grid, sizeof(T)));
    return launch_k(kern, grid, kMergeBlock, S::SMEM, ctx->stream, A->nsplit > 0, (int)A->n,
                    (const int *)A->rp.as<int>(), (const int *)A->col.as<int>(), val, x,
                    (const int2 *)A->tiles.as<int2>(), (int)A->ntiles, A->carry_row.as<int>(), A->carry_val.as<T>(),
                    A->flags.as<int>(), A->partials.as<T>(), A->ticket.as<unsigned>(), ctx->dev_err, e);
}

int ensure_hint(spx_ctx *ctx, spx_matrix *A, int ipt)
{
    if (A->hint.p && A->hint_ipt == ipt) return SPX_OK;
    const int64_t ng = ceil_div(A->nnz, ipt);
    dbuf_free(ctx, A->hint);
    SPX_TRY(dbuf_alloc(ctx, A->hint, (size_t)(ng > 0 ? ng : 1) * 4));
    if (ng > 0) {
        k_row_hint<<<(int)ceil_div(ng, 256), 256, 0, ctx->stream>>>((int)A->n, (int)A->nnz, A->rp.as<int>(), ipt,
                                                                  (int)ng, A->hint.as<int>());
        SPX_CUDA(cudaGetLastError());
    }
    A->hint_ipt = ipt;
    return SPX_OK;
}

// y = A x with nothing else: no scaling, no z, no dots
template <class T> bool epi_is_plain(const Epi<T> &e)
{
    return e.alpha == T(1) && !e.z && !e.w && !e.want_yy && !e.dots;
}

// Compile-time epilogue (see out_row): 1 plain, 4-7 the solvers' forms, 0
// anything else.
template <class T> int epi_mode(const Epi<T> &e)
{
    if (epi_is_plain(e)) return 1;
    if (!e.dots) return 0;
    if (e.alpha == T(1) && !e.z) {
        if (e.w) return e.want_yy ? 5 : 4;
        if (e.want_yy) return 6;
    }
    if (e.alpha == T(-1) && e.beta == T(1) && e.z && !e.w && e.want_yy) return 7;
    return 0;
}

constexpr int kRowsTile = 128;
constexpr int kRowsStages = 2;  // default shared-memory stages per block of the row-block kernel

int ensure_rows_cap(spx_ctx *ctx, spx_matrix *A)
{
    if (A->rows_cap >= 0) return SPX_OK;
    const int64_t ntiles = ceil_div(A->n, kRowsTile);
    DBuf m;
    SPX_TRY(dbuf_alloc(ctx, m, 16));
    int cap = 0;
    cudaError_t e = cudaMemsetAsync(m.p, 0, 4, ctx->stream);
    if (e == cudaSuccess && ntiles > 0) {
        const int g = (int)std::min<int64_t>(ceil_div(ntiles, 256), (int64_t)ctx->grid_sms * 8);
        k_tile_max_nnz<<<g, 256, 0, ctx->stream>>>((int)A->n, A->rp.as<int>(), kRowsTile, (int)ntiles, m.as<int>());
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cap, m.p, 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dbuf_free(ctx, m);
    if (e != cudaSuccess) return cuda_fail(e, "row-block tile sizes");
    A->rows_cap = cap;
    return SPX_OK;
}

// shared memory the row-block kernel needs for A (bytes)
template <class T> int64_t rows_smem(const spx_matrix *A, int stages)
{
    return RowsShape<T, kRowsTile>::smem((int)std::min<int64_t>(A->rows_cap, 1 << 24), stages);
}

template <class T, int STAGES, int MODE, int TPR>
int launch_rows_m(spx_ctx *ctx, spx_matrix *A, const T *val, const T *x, const Epi<T> &e)
{
    auto kern = k_csr_rows<T, kRowsTile, STAGES, MODE, TPR>;
    constexpr int block = kRowsTile * TPR;
    SPX_TRY(ensure_rows_cap(ctx, A));
    // the dynamic shared memory may reach the opt-in limit less the static part
    int dyn_max = 0;
    SPX_TRY(smem_optin(reinterpret_cast<const void *>(kern), -1, &dyn_max));
    const int64_t smem = rows_smem<T>(A, STAGES);
    if (smem > dyn_max)
        return fail(SPX_ERR_TOO_LARGE, "row-block CSR: a tile of 128 rows does not fit in shared memory");
    const int64_t ntiles = ceil_div(A->n, kRowsTile);
    const int grid = grid_for(ctx, kern, block, (int)smem, ntiles);
    SPX_TRY(ensure_scratch(ctx, A, 0, grid, sizeof(T)));
    kern<<<grid, block, (int)smem, ctx->stream>>>((int)A->n, A->rp.as<int>(), A->col.as<int>(), val, x,
                                                      (int)ntiles, (int)A->rows_cap, A->partials.as<T>(),
                                                      A->ticket.as<unsigned>(), ctx->dev_err, e);
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

// Threads per row when the caller leaves it open.  Rows of 16 or more entries
// make a 128-row tile large enough that only two tiles stay resident per SM,
// and one thread per row then leaves too few gathers in flight: two threads per
// row for FP64, four for FP32 (measured best on the 27-point stencil, 100^3:
// 88.7 -> 80.5 us FP64, 51.9 -> 47.8 us FP32).  Shorter rows keep one thread
// (the 7-point stencil, 128^3, FP64: 45.7 us with one, 70.3 us with two).
template <class T> int rows_auto_tpr(const spx_matrix *A)
{
    return A->mean_len < 16.0 ? 1 : sizeof(T) == 4 ? 4 : 2;
}

// stages: 1 or 2; tpr: threads per row, 1, 2 or 4 (2 and 4 with two stages only)
template <class T>
int launch_rows(spx_ctx *ctx, spx_matrix *A, const T *val, const T *x, const Epi<T> &e, int stages, int tpr)
{
#define SPX_ROWS_MODES(ST_, TPR_)                                             \
    switch (epi_mode(e)) {                                                    \
    case 1: return launch_rows_m<T, ST_, 1, TPR_>(ctx, A, val, x, e);         \
    case 4: return launch_rows_m<T, ST_, 4, TPR_>(ctx, A, val, x, e);         \
    case 5: return launch_rows_m<T, ST_, 5, TPR_>(ctx, A, val, x, e);         \
    case 6: return launch_rows_m<T, ST_, 6, TPR_>(ctx, A, val, x, e);         \
    case 7: return launch_rows_m<T, ST_, 7, TPR_>(ctx, A, val, x, e);         \
    default: return launch_rows_m<T, ST_, 0, TPR_>(ctx, A, val, x, e);        \
    }
    if (stages == 1) {
        if (tpr != 1) return fail(SPX_ERR_INVALID, "row-block CSR: several threads per row need two stages");
        SPX_ROWS_MODES(1, 1)
    }
    if (tpr == 2) {
        SPX_ROWS_MODES(2, 2)
    }
    if (tpr == 4) {
        SPX_ROWS_MODES(2, 4)
    }
    SPX_ROWS_MODES(2, 1)
#undef SPX_ROWS_MODES
}

int ensure_coo_rowtiles(spx_ctx *ctx, spx_matrix *A)
{
    if (A->coo_rows_cap >= 0) return SPX_OK;
    const int64_t ntiles = ceil_div(A->n, kRowsTile);
    if (ntiles + 1 > INT_MAX) return fail(SPX_ERR_TOO_LARGE, "too many COO row tiles");
    dbuf_free(ctx, A->coo_rowtiles);
    SPX_TRY(dbuf_alloc(ctx, A->coo_rowtiles, (size_t)(ntiles + 2) * 4 + 16));
    int *mx = A->coo_rowtiles.as<int>() + ntiles + 1;
    SPX_CUDA(cudaMemsetAsync(mx, 0, 4, ctx->stream));
    k_coo_rowtiles<<<(int)ceil_div(ntiles + 1, 256), 256, 0, ctx->stream>>>((int)A->n, A->coo_nnz, A->coo_row.as<int>(),
                                                                          kRowsTile, (int)ntiles,
                                                                          A->coo_rowtiles.as<int>(), mx);
    SPX_CUDA(cudaGetLastError());
    int cap = 0;
    SPX_CUDA(cudaMemcpyAsync(&cap, mx, 4, cudaMemcpyDeviceToHost, ctx->stream));
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    A->coo_rows_cap = cap;
    return SPX_OK;
}

template <class T> int64_t coo_rows_smem(const spx_matrix *A)
{
    return CooRowsShape<T, kRowsTile>::smem((int)std::min<int64_t>(A->coo_rows_cap, 1 << 24));
}

template <class T, int MODE>
int launch_coo_rows_m(spx_ctx *ctx, spx_matrix *A, const T *cval, const T *x, const Epi<T> &e)
{
    auto kern = k_coo_rows<T, kRowsTile, MODE>;
    SPX_TRY(ensure_coo_rowtiles(ctx, A));
    int dyn_max = 0;
    SPX_TRY(smem_optin(reinterpret_cast<const void *>(kern), -1, &dyn_max));
    const int64_t smem = coo_rows_smem<T>(A);
    if (smem > dyn_max)
        return fail(SPX_ERR_TOO_LARGE, "row-block COO: a tile of 128 rows does not fit in shared memory");
    const int64_t ntiles = ceil_div(A->n, kRowsTile);
    const int grid = grid_for(ctx, kern, kRowsTile, (int)smem, ntiles);
    SPX_TRY(ensure_scratch(ctx, A, 0, grid, sizeof(T)));
    kern<<<grid, kRowsTile, (int)smem, ctx->stream>>>((int)A->n, A->coo_row.as<int>(), A->coo_col.as<int>(), cval, x,
                                                      A->coo_rowtiles.as<int>(), (int)ntiles, (int)A->coo_rows_cap,
                                                      A->partials.as<T>(), A->ticket.as<unsigned>(), ctx->dev_err, e);
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

template <class T> int launch_coo_rows(spx_ctx *ctx, spx_matrix *A, const T *cval, const T *x, const Epi<T> &e)
{
    switch (epi_mode(e)) {
    case 1: return launch_coo_rows_m<T, 1>(ctx, A, cval, x, e);
    case 4: return launch_coo_rows_m<T, 4>(ctx, A, cval, x, e);
    case 5: return launch_coo_rows_m<T, 5>(ctx, A, cval, x, e);
    case 6: return launch_coo_rows_m<T, 6>(ctx, A, cval, x, e);
    case 7: return launch_coo_rows_m<T, 7>(ctx, A, cval, x, e);
    default: return launch_coo_rows_m<T, 0>(ctx, A, cval, x, e);
    }
}

template <class T, int IPT, int MODE>
int launch_split_m(spx_ctx *ctx, spx_matrix *A, const T *val, const T *x, const Epi<T> &e)
{
    auto kern = k_csr_split<T, IPT, MODE>;
    const int smem = 8 * (32 * IPT + 32) * (4 + (int)sizeof(T));
    SPX_TRY(set_smem(kern, smem));
    SPX_TRY(ensure_hint(ctx, A, IPT));
    const int64_t nchunks = ceil_div(ceil_div(A->nnz, IPT), 32);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * ctx->grid_sms;
    const int64_t need = ceil_div(nchunks, 8);  // at least one chunk per warp
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    SPX_TRY(ensure_scratch(ctx, A, grid * 8, grid, sizeof(T)));
    return launch_k(kern, (int)grid, 256, smem, ctx->stream, true, (int)A->n, (int)A->nnz, (const int *)A->rp.as<int>(),
                    (const int *)A->col.as<int>(), val, x, (const int *)A->hint.as<int>(), (int)nchunks,
                    A->carry_row.as<int>(), A->carry_val.as<T>(), A->flags.as<int>(), A->partials.as<T>(),
                    A->ticket.as<unsigned>(), ctx->dev_err, e);
}

template <class T, int IPT>
int launch_split(spx_ctx *ctx, spx_matrix *A, const T *val, const T *x, const Epi<T> &e)
{
    switch (epi_mode(e)) {
    case 1: return launch_split_m<T, IPT, 1>(ctx, A, val, x, e);
    case 4: return launch_split_m<T, IPT, 4>(ctx, A, val, x, e);
    case 5: return launch_split_m<T, IPT, 5>(ctx, A, val, x, e);
    case 6: return launch_split_m<T, IPT, 6>(ctx, A, val, x, e);
    case 7: return launch_split_m<T, IPT, 7>(ctx, A, val, x, e);
    default: return launch_split_m<T, IPT, 0>(ctx, A, val, x, e);
    }
}

// Tile-transposed nonzeros and granule descriptors for granules of ipt
// nonzeros (rebuilt when ipt changes); the values of `val` (the FP64 / FP32
// value array or the FP32 shadow) into the matching tiled buffer.
template <class T>
int ensure_tiled(spx_ctx *ctx, spx_matrix *A, int ipt, const T *val, const T **tval)
{
    const int64_t chunk = 32LL * ipt;
    const int64_t nchunks = ceil_div(A->nnz, chunk);
    const int64_t total = nchunks * chunk, ngran = nchunks * 32;
    if (ngran > INT_MAX / 2) return fail(SPX_ERR_TOO_LARGE, "tiled CSR: too many granules");
    if (A->tc_ipt != ipt) {
        dbuf_free(ctx, A->tc_col);
        dbuf_free(ctx, A->tc_row);
        dbuf_free(ctx, A->tc_mask);
        A->tc_val_ipt = A->tc_val32_ipt = 0;
        SPX_TRY(dbuf_alloc(ctx, A->tc_col, (size_t)total * 4 + 16));
        SPX_TRY(dbuf_alloc(ctx, A->tc_row, (size_t)(ngran + 1) * 4));
        SPX_TRY(dbuf_alloc(ctx, A->tc_mask, (size_t)(ngran + 1) * 4));
        k_tile_transpose<int, 4><<<(int)ceil_div(total, 256), 256, 0, ctx->stream>>>(
            A->nnz, total, ipt, A->col.as<int>(), A->tc_col.as<int>());
        SPX_CUDA(cudaGetLastError());
        k_tile_rows<<<(int)ceil_div(ngran + 1, 256), 256, 0, ctx->stream>>>(
            (int)A->n, A->nnz, A->rp.as<int>(), ipt, ngran, A->tc_row.as<int>(), A->tc_mask.as<unsigned>());
        SPX_CUDA(cudaGetLastError());
        k_tile_marks<<<(int)ceil_div(A->n, 256), 256, 0, ctx->stream>>>(
            (int)A->n, A->nnz, A->rp.as<int>(), ipt, A->tc_row.as<int>(), A->tc_mask.as<unsigned>());
        SPX_CUDA(cudaGetLastError());
        A->tc_ipt = ipt;
    }
    if (A->n_empty < 0) {  // the list of empty rows, once per matrix
        DBuf cnt;
        SPX_TRY(dbuf_alloc(ctx, cnt, 16));
        k_empty_rows<<<1, 1024, 0, ctx->stream>>>((int)A->n, A->rp.as<int>(), nullptr, cnt.as<int>());
        int h = 0;
        cudaError_t ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h, cnt.p, 4, cudaMemcpyDeviceToHost, ctx->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
        if (ce == cudaSuccess && h > 0) {
            const int st = dbuf_alloc(ctx, A->empty_rows, (size_t)h * 4);
            if (st != SPX_OK) {
                dbuf_free(ctx, cnt);
                return st;
            }
            k_empty_rows<<<1, 1024, 0, ctx->stream>>>((int)A->n, A->rp.as<int>(), A->empty_rows.as<int>(),
                                                      cnt.as<int>());
            ce = cudaGetLastError();
        }
        dbuf_free(ctx, cnt);
        if (ce != cudaSuccess) return cuda_fail(ce, "tiled CSR: empty-row list");
        A->n_empty = h;
    }
    const bool shadow = sizeof(T) == 4 && A->dtype == SPX_F64;  // the FP32 copy of FP64 values
    DBuf &tb = shadow ? A->tc_val32 : A->tc_val;
    int &tb_ipt = shadow ? A->tc_val32_ipt : A->tc_val_ipt;
    if (tb_ipt != ipt) {
        dbuf_free(ctx, tb);
        SPX_TRY(dbuf_alloc(ctx, tb, (size_t)total * sizeof(T) + 16));
        k_tile_transpose<T, 16 / (int)sizeof(T)><<<(int)ceil_div(total, 256), 256, 0, ctx->stream>>>(
            A->nnz, total, ipt, val, tb.as<T>());
        SPX_CUDA(cudaGetLastError());
        tb_ipt = ipt;
    }
    *tval = tb.as<T>();
    return SPX_OK;
}

template <class T, int IPT, int MODE>
int launch_tiled_m(spx_ctx *ctx, spx_matrix *A, const T *val, const T *x, const Epi<T> &e)
{
    auto kern = k_csr_tiled<T, IPT, MODE>;
    const T *tval = nullptr;
    SPX_TRY(ensure_tiled<T>(ctx, A, IPT, val, &tval));
    const int64_t nchunks = ceil_div(A->nnz, 32LL * IPT);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * ctx->grid_sms;
    const int64_t need = ceil_div(nchunks, 8);  // at least one chunk per warp
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    SPX_TRY(ensure_scratch(ctx, A, grid * 8, grid, sizeof(T)));
    return launch_k(kern, (int)grid, 256, 0, ctx->stream, true, (int)A->n, (int)A->nnz, (const int *)A->rp.as<int>(),
                    (const int *)A->tc_col.as<int>(), tval, (const int *)A->tc_row.as<int>(),
                    (const unsigned *)A->tc_mask.as<unsigned>(), (const int *)A->empty_rows.as<int>(),
                    (int)A->n_empty, x, (int)nchunks, A->carry_row.as<int>(), A->carry_val.as<T>(),
                    A->flags.as<int>(), A->partials.as<T>(), A->ticket.as<unsigned>(), ctx->dev_err, e);
}

template <class T, int IPT>
int launch_tiled(spx_ctx *ctx, spx_matrix *A, const T *val, const T *x, const Epi<T> &e)
{
    switch (epi_mode(e)) {
    case 1: return launch_tiled_m<T, IPT, 1>(ctx, A, val, x, e);
    case 4: return launch_tiled_m<T, IPT, 4>(ctx, A, val, x, e);
    case 5: return launch_tiled_m<T, IPT, 5>(ctx, A, val, x, e);
    case 6: return launch_tiled_m<T, IPT, 6>(ctx, A, val, x, e);
    case 7: return launch_tiled_m<T, IPT, 7>(ctx, A, val, x, e);
    default: return launch_tiled_m<T, IPT, 0>(ctx, A, val, x, e);
    }
}

// Tile-transposed copies of the COO arrays (row, column, values) for granules
// of ipt entries, rebuilt when ipt changes.
template <class T>
int ensure_coo_tiled(spx_ctx *ctx, spx_matrix *A, int ipt, const T *cval, const T **tval)
{
    const int64_t chunk = 32LL * ipt;
    const int64_t nchunks = ceil_div(A->coo_nnz, chunk);
    const int64_t total = nchunks * chunk;
    if (nchunks * 32 > INT_MAX / 2) return fail(SPX_ERR_TOO_LARGE, "tiled COO: too many granules");
    const int tb = (int)ceil_div(total, 256);
    if (A->ct_ipt != ipt) {
        dbuf_free(ctx, A->ct_row);
        dbuf_free(ctx, A->ct_col);
        A->ct_val_ipt = A->ct_val32_ipt = 0;
        SPX_TRY(dbuf_alloc(ctx, A->ct_row, (size_t)total * 4 + 16));
        SPX_TRY(dbuf_alloc(ctx, A->ct_col, (size_t)total * 4 + 16));
        k_tile_transpose<int, 4><<<tb, 256, 0, ctx->stream>>>(A->coo_nnz, total, ipt, A->coo_row.as<int>(),
                                                               A->ct_row.as<int>());
        k_tile_transpose<int, 4><<<tb, 256, 0, ctx->stream>>>(A->coo_nnz, total, ipt, A->coo_col.as<int>(),
                                                               A->ct_col.as<int>());
        SPX_CUDA(cudaGetLastError());
        A->ct_ipt = ipt;
    }
    const bool shadow = sizeof(T) == 4 && A->dtype == SPX_F64;
    DBuf &vb = shadow ? A->ct_val32 : A->ct_val;
    int &vb_ipt = shadow ? A->ct_val32_ipt : A->ct_val_ipt;
    if (vb_ipt != ipt) {
        dbuf_free(ctx, vb);
        SPX_TRY(dbuf_alloc(ctx, vb, (size_t)total * sizeof(T) + 16));
        k_tile_transpose<T, 16 / (int)sizeof(T)><<<tb, 256, 0, ctx->stream>>>(A->coo_nnz, total, ipt, cval,
                                                                               vb.as<T>());
        SPX_CUDA(cudaGetLastError());
        vb_ipt = ipt;
    }
    *tval = vb.as<T>();
    return SPX_OK;
}

template <class T, int IPT, int MODE>
int launch_coo_tiled_m(spx_ctx *ctx, spx_matrix *A, const T *cval, const T *x, const Epi<T> &e)
{
    auto kern = k_coo_tiled<T, IPT, MODE>;
    const T *tval = nullptr;
    SPX_TRY(ensure_coo_tiled<T>(ctx, A, IPT, cval, &tval));
    const int64_t nchunks = ceil_div(A->coo_nnz, 32LL * IPT);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * ctx->grid_sms;
    const int64_t need = ceil_div(nchunks, 8);
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    SPX_TRY(ensure_scratch(ctx, A, grid * 8, grid, sizeof(T)));
    return launch_k(kern, (int)grid, 256, 0, ctx->stream, true, (int)A->n, (int)A->coo_nnz,
                    (const int *)A->coo_row.as<int>(), (const int *)A->ct_row.as<int>(),
                    (const int *)A->ct_col.as<int>(), tval, x, (int)nchunks, A->carry_row.as<int>(),
                    A->carry_val.as<T>(), A->flags.as<int>(), A->partials.as<T>(), A->ticket.as<unsigned>(),
                    ctx->dev_err, e);
}

template <class T, int IPT>
int launch_coo_tiled(spx_ctx *ctx, spx_matrix *A, const T *cval, const T *x, const Epi<T> &e, int add)
{
    if (add) return e.alpha == T(1) ? launch_coo_tiled_m<T, IPT, 3>(ctx, A, cval, x, e)
                                    : launch_coo_tiled_m<T, IPT, 2>(ctx, A, cval, x, e);
    switch (epi_mode(e)) {
    case 1: return launch_coo_tiled_m<T, IPT, 1>(ctx, A, cval, x, e);
    case 4: return launch_coo_tiled_m<T, IPT, 4>(ctx, A, cval, x, e);
    case 5: return launch_coo_tiled_m<T, IPT, 5>(ctx, A, cval, x, e);
    case 6: return launch_coo_tiled_m<T, IPT, 6>(ctx, A, cval, x, e);
    case 7: return launch_coo_tiled_m<T, IPT, 7>(ctx, A, cval, x, e);
    default: return launch_coo_tiled_m<T, IPT, 0>(ctx, A, cval, x, e);
    }
}

template <class T, int IPT, int MODE>
int launch_coo_split_m(spx_ctx *ctx, spx_matrix *A, const T *cval, const T *x, const Epi<T> &e)
{
    auto kern = k_coo_split<T, IPT, MODE>;
    const int smem = 8 * (32 * IPT + 32) * (8 + (int)sizeof(T));
    SPX_TRY(set_smem(kern, smem));
    const int64_t nchunks = ceil_div(ceil_div(A->coo_nnz, IPT), 32);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * ctx->grid_sms;
    const int64_t need = ceil_div(nchunks, 8);
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    SPX_TRY(ensure_scratch(ctx, A, grid * 8, grid, sizeof(T)));
    return launch_k(kern, (int)grid, 256, smem, ctx->stream, true, (int)A->n, (int)A->coo_nnz,
                    (const int *)A->coo_row.as<int>(), (const int *)A->coo_col.as<int>(), cval, x, (int)nchunks,
                    A->carry_row.as<int>(), A->carry_val.as<T>(), A->flags.as<int>(), A->partials.as<T>(),
                    A->ticket.as<unsigned>(), ctx->dev_err, e);
}

// add: y += alpha A x (the COO part of HYB), else y = epilogue(A x)
template <class T, int IPT>
int launch_coo_split(spx_ctx *ctx, spx_matrix *A, const T *cval, const T *x, const Epi<T> &e, int add)
{
    if (add) return e.alpha == T(1) ? launch_coo_split_m<T, IPT, 3>(ctx, A, cval, x, e)
                                    : launch_coo_split_m<T, IPT, 2>(ctx, A, cval, x, e);
    switch (epi_mode(e)) {
    case 1: return launch_coo_split_m<T, IPT, 1>(ctx, A, cval, x, e);
    case 4: return launch_coo_split_m<T, IPT, 4>(ctx, A, cval, x, e);
    case 5: return launch_coo_split_m<T, IPT, 5>(ctx, A, cval, x, e);
    case 6: return launch_coo_split_m<T, IPT, 6>(ctx, A, cval, x, e);
    case 7: return launch_coo_split_m<T, IPT, 7>(ctx, A, cval, x, e);
    default: return launch_coo_split_m<T, IPT, 0>(ctx, A, cval, x, e);
    }
}

template <class T, int SW>
int launch_vector(spx_ctx *ctx, spx_matrix *A, const T *val, const T *x, const Epi<T> &e)
{
    auto kern = k_csr_vector<T, SW, kVecBlock>;
    const int64_t rows_per_block = (kVecBlock / 32) * (32 / SW);
    const int grid = grid_for(ctx, kern, kVecBlock, 0, ceil_div(A->n, rows_per_block));
    SPX_TRY(ensure_scratch(ctx, A, 0, grid, sizeof(T)));
    kern<<<grid, kVecBlock, 0, ctx->stream>>>(A->n, A->rp.as<int>(), A->col.as<int>(), val, x, e,
                                              A->partials.as<T>(), A->ticket.as<unsigned>());
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

template <class T, int R, int MODE>
int launch_ell_m(spx_ctx *ctx, spx_matrix *A, const T *eval, const T *x, const Epi<T> &e)
{
    auto kern = k_ell<T, R, kEllBlock, MODE>;
    const int grid = grid_for(ctx, kern, kEllBlock, 0, ceil_div(ceil_div(A->n, R), kEllBlock));
    SPX_TRY(ensure_scratch(ctx, A, 0, grid, sizeof(T)));
    kern<<<grid, kEllBlock, 0, ctx->stream>>>(A->n, A->ell_ld, (int)A->ell_w, A->ell_col.as<int>(),
                                              eval, x, e, A->partials.as<T>(),
                                              A->ticket.as<unsigned>());
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

// The plain-store mode pays off in FP32 (47.8 vs 50.7 us on the 27-point stencil);
// in FP64 it raises the kernel from 32 to 40 registers and the lost occupancy
// costs more (76.3 vs 70.2 us) than the epilogue's FP64 instructions save.
template <class T, int R>
int launch_ell(spx_ctx *ctx, spx_matrix *A, const T *eval, const T *x, const Epi<T> &e)
{
    switch (epi_mode(e)) {
    case 1: return sizeof(T) == 4 ? launch_ell_m<T, R, 1>(ctx, A, eval, x, e) : launch_ell_m<T, R, 0>(ctx, A, eval, x, e);
    case 4: return launch_ell_m<T, R, 4>(ctx, A, eval, x, e);
    case 5: return launch_ell_m<T, R, 5>(ctx, A, eval, x, e);
    case 6: return launch_ell_m<T, R, 6>(ctx, A, eval, x, e);
    case 7: return launch_ell_m<T, R, 7>(ctx, A, eval, x, e);
    default: return launch_ell_m<T, R, 0>(ctx, A, eval, x, e);
    }
}

template <class T, int IPT>
int launch_coo(spx_ctx *ctx, spx_matrix *A, const T *cval, const T *x, const Epi<T> &e, int add)
{
    using S = CooShape<T, kCooBlock, IPT>;
    auto kern = k_coo<T, kCooBlock, IPT>;
    SPX_TRY(set_smem(kern, S::SMEM));
    SPX_TRY(ensure_coo_tiles(ctx, A, S::TILE, S::SLACK));
    const int64_t ntiles = A->coo_ntiles;
    const int grid = grid_for(ctx, kern, kCooBlock, S::SMEM, ntiles);
    SPX_TRY(ensure_scratch(ctx, A, ntiles, grid, sizeof(T)));
    return launch_k(kern, grid, kCooBlock, S::SMEM, ctx->stream, A->coo_nsplit > 0, A->n, A->coo_nnz,
                    (const int *)A->coo_row.as<int>(), (const int *)A->coo_col.as<int>(), cval, x,
                    (const int *)A->coo_tiles.as<int>(), (int)ntiles, A->carry_row.as<int>(),
                    A->carry_val.as<T>(), A->flags.as<int>(), A->partials.as<T>(), A->ticket.as<unsigned>(),
                    ctx->dev_err, e, add);
}

template <class T> int launch_scale_only(spx_ctx *ctx, spx_matrix *A, const Epi<T> &e)
{
    auto kern = k_scale_only<T, 256>;
    const int grid = grid_for(ctx, kern, 256, 0, ceil_div(A->n, 256));
    SPX_TRY(ensure_scratch(ctx, A, 0, grid, sizeof(T)));
    kern<<<grid, 256, 0, ctx->stream>>>(A->n, e, A->partials.as<T>(), A->ticket.as<unsigned>());
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

template <class T> int launch_dots_of_y(spx_ctx *ctx, spx_matrix *A, const Epi<T> &e)
{
    auto kern = k_dots_of_y<T, 256>;
    const int grid = grid_for(ctx, kern, 256, 0, ceil_div(A->n, 256));
    SPX_TRY(ensure_scratch(ctx, A, 0, grid, sizeof(T)));
    kern<<<grid, 256, 0, ctx->stream>>>(A->n, e, A->partials.as<T>(), A->ticket.as<unsigned>());
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

template <class T>
int dispatch_csr(spx_ctx *ctx, spx_matrix *A, const T *val, const T *x, const Epi<T> &e)
{
    int kern = A->kernel, p = A->kparam;
    if (kern == SPX_KERNEL_AUTO) {
        // rows of nearly equal length: row blocks (one thread per row); moderately
        // uneven rows: merge-path tiles; heavy-tailed rows: the split kernel on the tiled copy
        // (2M-row power-law matrix, FP64: 156 us against 208 us for the split kernel staging
        // through shared memory)
        const double mx = (double)A->max_len, mean = A->mean_len;
        if (mx <= 2.0 * mean + 8.0) {
            SPX_TRY(ensure_rows_cap(ctx, A));
            if (rows_smem<T>(A, kRowsStages) <= std::min<int64_t>(ctx->max_smem_optin, 120 * 1024))
                return launch_rows<T>(ctx, A, val, x, e, kRowsStages, rows_auto_tpr<T>(A));
        }
        kern = mx <= 4.0 * mean + 8.0 ? SPX_KERNEL_CSR_MERGE : SPX_KERNEL_CSR_TILED;
        p = kern == SPX_KERNEL_CSR_TILED ? 32 : 0;
    }
    if (kern == SPX_KERNEL_CSR_ROWS) {  // param: stages + 10 x threads per row (0 = automatic)
        if (p == 0) return launch_rows<T>(ctx, A, val, x, e, kRowsStages, rows_auto_tpr<T>(A));
        if (p != 1 && p != 2 && p != 12 && p != 22 && p != 42)
            return fail(SPX_ERR_INVALID, "row-block parameter must be 0, 1, 2, 12, 22 or 42");
        return launch_rows<T>(ctx, A, val, x, e, p % 10, p < 10 ? 1 : p / 10);
    }
    if (kern == SPX_KERNEL_CSR_VECTOR) {
        if (p <= 0) {  // sub-warp width from the mean row length
            p = 1;
            while (p < 32 && p < A->mean_len) p <<= 1;
        }
        switch (p) {
        case 1: return launch_vector<T, 1>(ctx, A, val, x, e);
        case 2: return launch_vector<T, 2>(ctx, A, val, x, e);
        case 4: return launch_vector<T, 4>(ctx, A, val, x, e);
        case 8: return launch_vector<T, 8>(ctx, A, val, x, e);
        case 16: return launch_vector<T, 16>(ctx, A, val, x, e);
        case 32: return launch_vector<T, 32>(ctx, A, val, x, e);
        default: return fail(SPX_ERR_INVALID, "CSR vector sub-warp width must be 1..32, a power of 2");
        }
    }
    if (kern == SPX_KERNEL_CSR_SPLIT) {
        if (p <= 0) p = 16;
        switch (p) {
        case 8: return launch_split<T, 8>(ctx, A, val, x, e);
        case 16: return launch_split<T, 16>(ctx, A, val, x, e);
        default: return fail(SPX_ERR_INVALID, "split nonzeros per lane must be 8 or 16");
        }
    }
    if (kern == SPX_KERNEL_CSR_TILED) {
        if (p <= 0) p = 32;
        switch (p) {
        case 16: return launch_tiled<T, 16>(ctx, A, val, x, e);
        case 32: return launch_tiled<T, 32>(ctx, A, val, x, e);
        default: return fail(SPX_ERR_INVALID, "tiled CSR nonzeros per lane must be 16 or 32");
        }
    }
    if (kern == SPX_KERNEL_CSR_MERGE) {
        if (p <= 0) p = 8;
        switch (p) {
        case 4: return launch_merge<T, 4>(ctx, A, val, x, e);
        case 8: return launch_merge<T, 8>(ctx, A, val, x, e);
        case 16: return launch_merge<T, 16>(ctx, A, val, x, e);
        default: return fail(SPX_ERR_INVALID, "merge items per thread must be 4, 8 or 16");
        }
    }
    return fail(SPX_ERR_UNSUPPORTED, "kernel not valid for a CSR matrix");
}

template <class T>
int dispatch_ell(spx_ctx *ctx, spx_matrix *A, const T *eval, const T *x, const Epi<T> &e)
{
    int p = A->kernel == SPX_KERNEL_ELL ? A->kparam : 0;
    if (p <= 0) p = 2;  // two rows per thread (FP32 with four: 58.0 against 54.0 us on the 27-point stencil)
    if constexpr (sizeof(T) == 8) {
        if (p == 1) return launch_ell<T, 1>(ctx, A, eval, x, e);
        if (p == 2) return launch_ell<T, 2>(ctx, A, eval, x, e);
    } else {
        if (p == 1) return launch_ell<T, 1>(ctx, A, eval, x, e);
        if (p == 2) return launch_ell<T, 2>(ctx, A, eval, x, e);
        if (p == 4) return launch_ell<T, 4>(ctx, A, eval, x, e);
    }
    return fail(SPX_ERR_INVALID, "ELL rows per thread must be 1, 2 (FP64) or 1, 2, 4 (FP32)");
}

template <class T>
int dispatch_coo(spx_ctx *ctx, spx_matrix *A, const T *cval, const T *x, const Epi<T> &e, int add)
{
    // param: 1 = row-block (tiles of 128 rows, one thread per row; rows of similar length);
    // 8 / 16 = nonzeros per lane of the warp-independent split kernel;
    // 104 / 108 / 116 = tiled segmented reduction with 4 / 8 / 16 items per thread.
    // Default: row-block for the COO format with short rows of similar length (the
    // boundary scan of a tile costs about mean-row-length steps per thread: measured
    // faster than split for the 7-point stencil, slower for the 27-point one), else the
    // split kernel on tile-transposed copies with 16 entries per lane (FP64: 177 us on
    // the power-law matrix and 119 us on the 27-point stencil 100^3, against 208 and
    // 146 us for the split kernel staging through shared memory).
    int p = A->kernel == SPX_KERNEL_COO ? A->kparam : 0;
    if (p <= 0) {
        p = 216;
        if (!add && A->format == SPX_COO && A->mean_len <= 16.0 && (double)A->max_len <= 2.0 * A->mean_len + 8.0) {
            SPX_TRY(ensure_coo_rowtiles(ctx, A));
            if (coo_rows_smem<T>(A) <= std::min<int64_t>(ctx->max_smem_optin, 120 * 1024)) p = 1;
        }
    }
    if (p == 1) {
        if (add) return fail(SPX_ERR_UNSUPPORTED, "the row-block COO kernel does not run HYB's COO part");
        return launch_coo_rows<T>(ctx, A, cval, x, e);
    }
    switch (p) {
    case 216: return launch_coo_tiled<T, 16>(ctx, A, cval, x, e, add);
    case 232: return launch_coo_tiled<T, 32>(ctx, A, cval, x, e, add);
    case 8: return launch_coo_split<T, 8>(ctx, A, cval, x, e, add);
    case 16: return launch_coo_split<T, 16>(ctx, A, cval, x, e, add);
    case 104: return launch_coo<T, 4>(ctx, A, cval, x, e, add);
    case 108: return launch_coo<T, 8>(ctx, A, cval, x, e, add);
    case 116: return launch_coo<T, 16>(ctx, A, cval, x, e, add);
    default:
        return fail(SPX_ERR_INVALID,
                    "COO kernel parameter must be 1 (row-block), 8, 16 (split), 216, 232 (tiled split) or 104, 108, "
                    "116 (tiled segmented reduction)");
    }
}

}  // namespace

int ensure_merge_tiles(spx_ctx *ctx, spx_matrix *A, int64_t tile_items, int64_t slack)
{
    if (A->tiles.p && A->tiles_items == tile_items) return SPX_OK;
    const int64_t items = A->n + A->nnz;
    const int64_t ntiles = ceil_div(items, tile_items);
    if (ntiles + 1 > INT_MAX) return fail(SPX_ERR_TOO_LARGE, "too many merge tiles");
    dbuf_free(ctx, A->tiles);
    SPX_TRY(dbuf_alloc(ctx, A->tiles, (size_t)(ntiles + 1) * sizeof(int2) + 16));
    unsigned *cnt = reinterpret_cast<unsigned *>(A->tiles.as<int2>() + ntiles + 1);
    SPX_CUDA(cudaMemsetAsync(cnt, 0, 4, ctx->stream));
    const int threads = 256;
    k_merge_tiles<<<(int)ceil_div(ntiles + 1, threads), threads, 0, ctx->stream>>>(
        (int)A->n, (int)A->nnz, A->rp.as<int>(), tile_items, slack, (int)ntiles, A->tiles.as<int2>(), cnt);
    SPX_CUDA(cudaGetLastError());
    unsigned h = 0;
    SPX_CUDA(cudaMemcpyAsync(&h, cnt, 4, cudaMemcpyDeviceToHost, ctx->stream));
    SPX_CUDA(cudaStreamSynchronize(ctx->stream));
    A->tiles_items = tile_items;
    A->ntiles = ntiles;
    A->nsplit = h;
    return SPX_OK;
}

template <class T>
int spmv_launch(spx_ctx *ctx, const spx_matrix *Ac, const T *x, const Epi<T> &e, bool use32)
{
    spx_matrix *A = const_cast<spx_matrix *>(Ac);
    if (A->n == 0) return SPX_OK;
    auto pick = [&](const spx::DBuf &v64, const spx::DBuf &v32) -> const T * {
        return static_cast<const T *>(use32 ? v32.p : v64.p);
    };
    switch (A->format) {
    case SPX_CSR:
        if (A->nnz == 0) return launch_scale_only<T>(ctx, A, e);
        return dispatch_csr<T>(ctx, A, pick(A->val, A->val32), x, e);
    case SPX_ELL:
        if (A->ell_w == 0) return launch_scale_only<T>(ctx, A, e);
        return dispatch_ell<T>(ctx, A, pick(A->ell_val, A->ell_val32), x, e);
    case SPX_COO:
        if (A->coo_nnz == 0) return launch_scale_only<T>(ctx, A, e);
        return dispatch_coo<T>(ctx, A, pick(A->coo_val, A->coo_val32), x, e, 0);
    case SPX_HYB: {
        Epi<T> first = e;
        first.dots = nullptr;
        first.fin = FIN_NONE;
        first.w = nullptr;
        first.want_yy = false;
        if (A->ell_w > 0) SPX_TRY(dispatch_ell<T>(ctx, A, pick(A->ell_val, A->ell_val32), x, first));
        else SPX_TRY(launch_scale_only<T>(ctx, A, first));
        if (A->coo_nnz > 0) {
            Epi<T> add = first;
            add.z = nullptr;
            SPX_TRY(dispatch_coo<T>(ctx, A, pick(A->coo_val, A->coo_val32), x, add, 1));
        }
        if (e.dots) SPX_TRY(launch_dots_of_y<T>(ctx, A, e));
        return SPX_OK;
    }
    default: return fail(SPX_ERR_INVALID, "unknown matrix format");
    }
}

template int spmv_launch<double>(spx_ctx *, const spx_matrix *, const double *, const Epi<double> &, bool);
template int spmv_launch<float>(spx_ctx *, const spx_matrix *, const float *, const Epi<float> &, bool);

}  // namespace spx

// ------------------------------------------------------------------ SpMV without allocation
// Some callers cannot allocate device memory at the point where they need a
// product: a real-time loop whose memory is fixed up front (an allocation can
// block, fail or synchronise the device), or a host framework that owns every
// allocation and forbids libraries from calling cudaMalloc.  For them this
// entry point runs the merge-path
// CSR kernel straight from the caller's CSR arrays with all of its scratch
// (tile map, per-tile carries, look-back flags) in one fixed array in device
// global memory that the library declares at file scope.  Every GPU that
// loads the library holds that array until the process exits.
namespace spx {
namespace {

constexpr int kNoAllocIpt = 8;
constexpr int64_t kNoAllocMaxTiles = SPX_NOALLOC_MAX_TILES;
constexpr size_t kNoAllocBytes = 1u << 20;  // 1 MiB

// scratch layout: tiles int2[max+1] | carry_val 8B[max] | carry_row int[max] | flags int[max] | counters,
// and the error word of the bounded waits in the last 64 bytes
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
static_assert((kNoAllocMaxTiles + 1) * 8 + kNoAllocMaxTiles * (8 + 4 + 4) + 256 <= (int64_t)kNoAllocBytes,
              "no-alloc scratch too small for its tile limit");

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[256];  // device address of the scratch per device, set once

int noalloc_scratch(int dev, void **out)
{
    if (dev < 0 || dev >= 256) return fail(SPX_ERR_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        // host code must not use the symbol itself: it names a host-side stand-in
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return SPX_OK;
}

// After the product: if any bounded wait of this call gave up (its bit is in
// *err, cleared at the start of the call), y is not the product, and every
// element becomes NaN so the caller sees the failure in the result itself.
template <class T> __global__ void __launch_bounds__(256) k_noalloc_poison(const unsigned *err, int64_t n, T *y)
{
    if (ldcg(err) == 0u) return;
    const T nan = T(NAN);
    for (int64_t i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) y[i] = nan;
}

template <class T>
int spmv_noalloc(cudaStream_t st, void *scratch, int64_t n, int64_t nnz, const int *rp, const int *col, const T *val,
                 const T *x, T *y, int sm_count, unsigned *err)
{
    using S = MergeShape<T, kMergeBlock, kNoAllocIpt>;
    auto kern = k_csr_merge<T, kMergeBlock, kNoAllocIpt>;
    const int64_t ntiles = ceil_div(n + nnz, S::TILE);
    char *base = static_cast<char *>(scratch);
    int2 *tiles = reinterpret_cast<int2 *>(base);
    T *carry_val = reinterpret_cast<T *>(base + (kNoAllocMaxTiles + 1) * 8);
    int *carry_row = reinterpret_cast<int *>(base + (kNoAllocMaxTiles + 1) * 8 + kNoAllocMaxTiles * 8);
    int *flags = carry_row + kNoAllocMaxTiles;
    unsigned *counters = reinterpret_cast<unsigned *>(flags + kNoAllocMaxTiles);  // nsplit, ticket
    // the array keeps the previous call's contents: flags and counters must start at zero
    SPX_CUDA(cudaMemsetAsync(flags, 0, (size_t)ntiles * 4, st));
    SPX_CUDA(cudaMemsetAsync(counters, 0, 64, st));
    SPX_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
    k_merge_tiles<<<(int)ceil_div(ntiles + 1, 256), 256, 0, st>>>((int)n, (int)nnz, rp, S::TILE, S::SLACK, (int)ntiles,
                                                                 tiles, counters);
    SPX_CUDA(cudaGetLastError());
    SPX_TRY(set_smem(kern, S::SMEM));
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMergeBlock, S::SMEM) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t grid = (int64_t)per_sm * sm_count;
    if (grid > ntiles) grid = ntiles;
    Epi<T> e;
    e.y = y;
    // the split count is not read back (no synchronisation): always launch cooperatively
    SPX_TRY(launch_k(kern, (int)grid, kMergeBlock, S::SMEM, st, true, (int)n, rp, col, val, x, (const int2 *)tiles,
                     (int)ntiles, carry_row, carry_val, flags, (T *)nullptr, counters + 1, err, e));
    const int pgrid = (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)sm_count * 4);
    k_noalloc_poison<T><<<pgrid, 256, 0, st>>>(err, n, y);
    SPX_CUDA(cudaGetLastError());
    return SPX_OK;
}

}  // namespace
}  // namespace spx

extern "C" int spx_spmv_csr_noalloc(void *stream, int dtype, int64_t nrows, int64_t ncols, int64_t nnz,
                                    const int32_t *row_ptr, const int32_t *col_idx, const void *values,
                                    const void *x, void *y)
{
    using namespace spx;
    if (dtype != SPX_F64 && dtype != SPX_F32) return fail(SPX_ERR_INVALID, "spx_spmv_csr_noalloc: bad dtype");
    if (nrows < 0 || ncols < 0 || nnz < 0 || nrows >= INT_MAX || nnz > INT_MAX)
        return fail(SPX_ERR_INVALID, "spx_spmv_csr_noalloc: bad sizes");
    if (nrows == 0) return SPX_OK;
    if (!row_ptr || !y || (nnz > 0 && (!col_idx || !values || !x)))
        return fail(SPX_ERR_INVALID, "spx_spmv_csr_noalloc: NULL array");
    const int64_t tile = (int64_t)kMergeBlock * kNoAllocIpt;
    if (ceil_div(nrows + nnz, tile) > kNoAllocMaxTiles)
        return fail(SPX_ERR_TOO_LARGE, "spx_spmv_csr_noalloc: nrows + nnz = " + std::to_string((long long)(nrows + nnz)) +
                                           " exceeds the fixed scratch limit of " +
                                           std::to_string((long long)(kNoAllocMaxTiles * tile)));
    if (((uintptr_t)row_ptr | (uintptr_t)col_idx | (uintptr_t)values) & 15u)
        return fail(SPX_ERR_INVALID, "spx_spmv_csr_noalloc: row_ptr, col_idx and values must be 16-byte aligned");
    int dev = 0;
    SPX_CUDA(cudaGetDevice(&dev));
    void *scratch = nullptr;
    SPX_TRY(noalloc_scratch(dev, &scratch));
    int sms = 0;
    SPX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned *err = reinterpret_cast<unsigned *>(static_cast<char *>(scratch) + kNoAllocBytes - 64);
    if (nnz == 0) {  // y = 0
        const cudaError_t e = cudaMemsetAsync(y, 0, (size_t)nrows * (dtype == SPX_F64 ? 8 : 4), st);
        return e == cudaSuccess ? SPX_OK : cuda_fail(e, "cudaMemsetAsync");
    }
    if (dtype == SPX_F64)
        return spmv_noalloc<double>(st, scratch, nrows, nnz, row_ptr, col_idx, static_cast<const double *>(values),
                                    static_cast<const double *>(x), static_cast<double *>(y), sms, err);
    return spmv_noalloc<float>(st, scratch, nrows, nnz, row_ptr, col_idx, static_cast<const float *>(values),
                               static_cast<const float *>(x), static_cast<float *>(y), sms, err);
}

// ------------------------------------------------------------------ gather probe
// A measurement aid, not part of SpMV: the part of a CSR / COO SpMV that no
// kernel can avoid for a given sparsity pattern — stream the column indices
// and gather x at each of them — with no values, rows or arithmetic beyond a
// running sum (kept so the gathers are not optimised away).  Its time is a
// floor for any SpMV kernel on that pattern.
namespace {
template <class T>
__global__ void __launch_bounds__(256)
    k_gather_probe(int64_t nnz, const int *__restrict__ col, const T *__restrict__ x, T *__restrict__ out)
{
    T acc = T(0);
    const int64_t stride = (int64_t)gridDim.x * 256;
    int64_t k = blockIdx.x * 256LL + threadIdx.x;
    for (; k + 7 * stride < nnz; k += 8 * stride) {  // eight gathers in flight per thread
        int c[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) c[u] = col[k + u * stride];
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldg(x + c[u]);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
    }
    for (; k < nnz; k += stride) acc += __ldg(x + col[k]);
    acc = spx::warp_sum(acc);
    if ((threadIdx.x & 31) == 0 && acc == T(-12345.678)) out[0] = acc;  // practically never stores
}
}  // namespace

extern "C" int spx_probe_gather(spx_ctx *ctx, int64_t nnz, const int32_t *col_idx, const void *x, int dtype,
                                void *out)
{
    if (!ctx || nnz < 0 || (nnz > 0 && (!col_idx || !x || !out))) return spx::fail(SPX_ERR_INVALID, "spx_probe_gather: bad argument");
    if (dtype != SPX_F64 && dtype != SPX_F32) return spx::fail(SPX_ERR_INVALID, "spx_probe_gather: bad dtype");
    if (nnz == 0) return SPX_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    const int grid = ctx->grid_sms * 8;
    if (dtype == SPX_F64)
        k_gather_probe<double><<<grid, 256, 0, ctx->stream>>>(nnz, col_idx, static_cast<const double *>(x),
                                                             static_cast<double *>(out));
    else
        k_gather_probe<float><<<grid, 256, 0, ctx->stream>>>(nnz, col_idx, static_cast<const float *>(x),
                                                            static_cast<float *>(out));
    const cudaError_t e = cudaGetLastError();
    if (prev != ctx->device) cudaSetDevice(prev);
    return e == cudaSuccess ? SPX_OK : spx::cuda_fail(e, "spx_probe_gather");
}

// ------------------------------------------------------------------ bounded-wait self-test
// A test hook for the failure path: one warp waits, with a short limit, on a
// look-back flag (which = 0) or an mbarrier phase (which = 1) that nothing
// will ever complete.  The wait gives up, records the error bit in the
// context's error word and the kernel returns normally; spx_ctx_check then
// reports SPX_ERR_TIMEOUT.  Nothing hangs and nothing faults.
namespace {
__global__ void k_selftest_wait(int which, long long limit_cycles, int *never_set, unsigned *err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    if (which == 0) {
        spx::flag_wait(never_set, err, limit_cycles);
    } else {
        spx::mbar_init(&bar, 1);
        spx::fence_barrier_init();
        spx::mbar_wait(&bar, 0, err, limit_cycles);  // phase 0 never completes: nobody arrives
    }
}
}  // namespace

extern "C" int spx_selftest_wait_timeout(spx_ctx *ctx, int which)
{
    if (!ctx || (which != 0 && which != 1)) return spx::fail(SPX_ERR_INVALID, "spx_selftest_wait_timeout: bad argument");
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    int *flag = nullptr;
    cudaError_t e = cudaMallocAsync(&flag, 16, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, 16, ctx->stream);
    if (e == cudaSuccess) {
        k_selftest_wait<<<1, 32, 0, ctx->stream>>>(which, 2000000LL, flag, ctx->dev_err);  // about 1 ms
        e = cudaGetLastError();
    }
    if (flag) cudaFreeAsync(flag, ctx->stream);
    if (prev != ctx->device) cudaSetDevice(prev);
    return e == cudaSuccess ? SPX_OK : spx::cuda_fail(e, "spx_selftest_wait_timeout");
}
