// efm_flux.cu -- exact flux vectors of results (Def. 3).
//
// For a support U with nullity(S_int[:, U]) = 1 the balanced flux modes on
// U form one ray: the kernel of S_int[:, U].  One warp per support streams
// the rows of S_int that U touches and keeps an integer basis of the row
// space in reduced echelon form (every basis row is zero in the other rows'
// pivot columns), built by cross-multiplication and division by the row's
// gcd, so it stays exact and small.  With n columns and rank n - 1 the one
// free column f gives the kernel vector: x_f = lcm of the pivots, x_p =
// -B[f] x_f / B[p] for each basis row; then divided by the gcd and oriented
// positive.  Products are formed in 128 bits and must fit in 64.
#include "efm_internal.cuh"

namespace efm {

namespace {

constexpr unsigned FULLM = 0xFFFFFFFFu;
constexpr int kFluxWarps = 4;
constexpr int kFluxMaxCols = 64;

struct FluxWarpSmem {
    int64_t B[kFluxMaxCols - 1][kFluxMaxCols];  // basis rows
    int piv[kFluxMaxCols];                      // pivot column of each basis row
    int cols[kFluxMaxCols];                     // the support's columns, ascending
    uint32_t rows[EFM_MAX_INTERNAL / 32];       // internal rows touched by the support
};

__device__ __forceinline__ uint64_t uabs(int64_t x) { return x < 0 ? 0ull - (uint64_t)x : (uint64_t)x; }

__device__ __forceinline__ uint64_t gcd_u(uint64_t a, uint64_t b)
{
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

__device__ __forceinline__ bool fits64(__int128 v)
{
    return v >= (__int128)INT64_MIN && v <= (__int128)INT64_MAX;
}

// a * x - b * y in 128 bits; false when it leaves int64
__device__ __forceinline__ bool cross(int64_t a, int64_t x, int64_t b, int64_t y, int64_t &out)
{
    const __int128 v = (__int128)a * x - (__int128)b * y;
    out = (int64_t)v;
    return fits64(v);
}

// divide the warp's row (two entries per lane) by the gcd of its entries
__device__ __forceinline__ void make_primitive(int64_t &x0, int64_t &x1)
{
    uint64_t g = gcd_u(uabs(x0), uabs(x1));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) g = gcd_u(g, __shfl_xor_sync(FULLM, g, off));
    if (g > 1) {
        x0 /= (int64_t)g;
        x1 /= (int64_t)g;
    }
}

__global__ void __launch_bounds__(kFluxWarps * 32) flux_kernel(NetView nv, const uint64_t *sup, int64_t n, int64_t *flux,
                                                              int8_t *status)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    FluxWarpSmem &S = reinterpret_cast<FluxWarpSmem *>(fsm)[wid];
    const uint32_t *bl = nv.blob;
    const int32_t *dcol = reinterpret_cast<const int32_t *>(bl + nv.o_dcols);
    const int W = nv.W, Mw = (nv.M + 31) / 32;
    for (int64_t r = (int64_t)blockIdx.x * kFluxWarps + wid; r < n; r += (int64_t)gridDim.x * kFluxWarps) {
        const uint64_t *U = sup + (size_t)r * W;
        // the columns of U in ascending order
        int nc = 0;
        for (int w0 = 0; w0 < W; w0 += 32) {
            const uint64_t x = w0 + lane < W ? U[w0 + lane] : 0ull;
            const int c = __popcll(x);
            int incl = c;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(FULLM, incl, off);
                if (lane >= off) incl += y;
            }
            int pos = nc + incl - c;
            uint64_t y = x;
            while (y) {
                const int b = __ffsll((long long)y) - 1;
                y &= y - 1;
                if (pos < kFluxMaxCols) S.cols[pos] = (w0 + lane) * 64 + b;
                ++pos;
            }
            nc += __shfl_sync(FULLM, incl, 31);
        }
        int8_t st = 1;
        if (nc < 1 || nc > kFluxMaxCols) st = -1;
        for (int w = lane; w < Mw; w += 32) S.rows[w] = 0u;
        __syncwarp();
        if (st == 1) {
            for (int j = lane; j < nc; j += 32) {
                const int c = S.cols[j];
                for (int q = (int)bl[nv.o_colptr + c]; q < (int)bl[nv.o_colptr + c + 1]; ++q) {
                    const int m = ent_index(bl[nv.o_colent + q]);
                    atomicOr(&S.rows[m >> 5], 1u << (m & 31));
                }
            }
        }
        __syncwarp();
        int nb = 0;
        bool ovf = false;
        const int j0 = lane, j1 = lane + 32;
        for (int w = 0; w < Mw && st == 1 && !ovf; ++w) {
            uint32_t bits = S.rows[w];
            while (bits && st == 1 && !ovf) {
                const int m = w * 32 + __ffs((int)bits) - 1;
                bits &= bits - 1;
                int64_t x0 = j0 < nc ? dcol[(size_t)S.cols[j0] * nv.Mpad + m] : 0;
                int64_t x1 = j1 < nc ? dcol[(size_t)S.cols[j1] * nv.Mpad + m] : 0;
                // reduce by every basis row
                for (int k = 0; k < nb && !ovf; ++k) {
                    const int p = S.piv[k];
                    const int64_t xp = __shfl_sync(FULLM, p < 32 ? x0 : x1, p & 31);
                    if (xp == 0) continue;
                    const int64_t bp = S.B[k][p];
                    bool ok = cross(bp, x0, xp, j0 < nc ? S.B[k][j0] : 0, x0);
                    ok = cross(bp, x1, xp, j1 < nc ? S.B[k][j1] : 0, x1) && ok;
                    ovf = __any_sync(FULLM, !ok);
                    make_primitive(x0, x1);
                }
                if (ovf) break;
                const unsigned m0 = __ballot_sync(FULLM, x0 != 0), m1 = __ballot_sync(FULLM, x1 != 0);
                if (!m0 && !m1) continue;  // dependent row
                const int p = m0 ? __ffs((int)m0) - 1 : 32 + __ffs((int)m1) - 1;
                if (nb == nc - 1) {
                    st = -1;  // rank n: no kernel
                    break;
                }
                int64_t xp = __shfl_sync(FULLM, p < 32 ? x0 : x1, p & 31);
                if (xp < 0) {
                    x0 = -x0;
                    x1 = -x1;
                    xp = -xp;
                }
                // clear column p from the basis (reduced form)
                for (int k = 0; k < nb && !ovf; ++k) {
                    const int64_t bk = S.B[k][p];
                    __syncwarp();
                    if (bk == 0) continue;
                    int64_t y0 = j0 < nc ? S.B[k][j0] : 0, y1 = j1 < nc ? S.B[k][j1] : 0;
                    bool ok = cross(xp, y0, bk, x0, y0);
                    ok = cross(xp, y1, bk, x1, y1) && ok;
                    ovf = __any_sync(FULLM, !ok);
                    make_primitive(y0, y1);
                    __syncwarp();
                    if (j0 < nc) S.B[k][j0] = y0;
                    if (j1 < nc) S.B[k][j1] = y1;
                }
                __syncwarp();
                if (j0 < nc) S.B[nb][j0] = x0;
                if (j1 < nc) S.B[nb][j1] = x1;
                if (lane == 0) S.piv[nb] = p;
                ++nb;
                __syncwarp();
            }
        }
        if (st == 1 && !ovf && nb != nc - 1) st = -1;
        int64_t v0 = 0, v1 = 0;
        if (st == 1 && !ovf) {
            // the free column: the one column without a pivot
            const bool p0 = j0 < nc, p1 = j1 < nc;
            bool hp0 = false, hp1 = false;
            for (int k = 0; k < nb; ++k) {
                hp0 = hp0 || S.piv[k] == j0;
                hp1 = hp1 || S.piv[k] == j1;
            }
            const unsigned f0 = __ballot_sync(FULLM, p0 && !hp0), f1 = __ballot_sync(FULLM, p1 && !hp1);
            const int f = f0 ? __ffs((int)f0) - 1 : 32 + __ffs((int)f1) - 1;
            // x_f = lcm of |pivots| (lane 0), x_p = -B[f] x_f / B[p]
            int64_t L = 1;
            if (lane == 0) {
                for (int k = 0; k < nb && !ovf; ++k) {
                    const uint64_t a = uabs(S.B[k][S.piv[k]]);
                    const uint64_t g = gcd_u((uint64_t)L, a);
                    const __int128 l = (__int128)(L / (int64_t)g) * (__int128)a;
                    ovf = !fits64(l);
                    L = (int64_t)l;
                }
            }
            ovf = __shfl_sync(FULLM, ovf ? 1 : 0, 0) != 0;
            L = __shfl_sync(FULLM, L, 0);
            if (!ovf) {
                bool ok = true;
                for (int k = 0; k < nb; ++k) {
                    const int p = S.piv[k];
                    if ((p & 31) != lane) continue;
                    const __int128 v = -(__int128)S.B[k][f] * (__int128)(L / S.B[k][p]);
                    ok = ok && fits64(v);
                    if (p < 32)
                        v0 = (int64_t)v;
                    else
                        v1 = (int64_t)v;
                }
                if (f == j0) v0 = L;
                if (f == j1) v1 = L;
                ovf = __any_sync(FULLM, !ok);
            }
            if (!ovf) {
                make_primitive(v0, v1);
                const bool bad = (p0 && v0 <= 0) || (p1 && v1 <= 0);
                if (__any_sync(FULLM, bad)) st = -1;
            }
        }
        if (ovf && st == 1) st = 0;
        int64_t *out = flux + (size_t)r * kFluxMaxCols;
        out[j0] = st == 1 ? v0 : 0;
        out[j1] = st == 1 ? v1 : 0;
        if (lane == 0) status[r] = st;
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_flux(const NetView &nv, const uint64_t *sup, int64_t n, int64_t *flux, int8_t *status, int sm_count,
                        cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(FluxWarpSmem) * kFluxWarps;
    cudaFuncSetAttribute(flux_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = (int)std::min<int64_t>((n + kFluxWarps - 1) / kFluxWarps, (int64_t)sm_count);
    flux_kernel<<<grid, kFluxWarps * 32, smem, s>>>(nv, sup, n, flux, status);
    return cudaGetLastError();
}

}  // namespace efm
