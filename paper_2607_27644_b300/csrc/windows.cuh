// Sliding-window decoding with a commit region of one round (arXiv
// 2607.27644, Sec. 6.1, decoding-latency paragraph: about d rounds of
// syndromes are decoded every syndrome-extraction round).  The windows
// themselves decode with the ordinary Relay-BP kernels, each on its own
// handle built from the DEM restricted to the window's rows and columns; the
// kernels here move syndromes and corrections between the windows:
//
//   window t: rows of rounds [t, t + w), columns whose earliest detector lies
//   in those rounds; decode the residual syndrome r on the window's rows;
//   commit the columns of round t (every column of the last window): their
//   bits join e^ and their detector sets are XORed into r, which clears round
//   t whenever the window converged.
#pragma once
#include "kernels.cuh"

namespace relaybp {

// Window syndromes: bit k of shot s = bit rows[k] of the residual.  One thread
// per (shot, output word).
__global__ void win_gather_kernel(const uint32_t *__restrict__ resid, int wcf, const int32_t *__restrict__ rows,
                                  int nrows, uint32_t *__restrict__ wsyn, int wcw, int64_t shots)
{
    const int64_t total = shots * (int64_t)wcw;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = q / wcw;
        const int w = (int)(q % wcw);
        const uint32_t *r = resid + s * wcf;
        uint32_t word = 0u;
        const int k1 = min(32, nrows - w * 32);
        for (int b = 0; b < k1; ++b) {
            const int i = __ldg(rows + w * 32 + b);
            word |= ((r[i >> 5] >> (i & 31)) & 1u) << b;
        }
        wsyn[q] = word;
    }
}

// Commit: for each committed column (window index lc, DEM index jf) whose bit
// is set in the window's correction, set bit jf of e^ and flip its detectors
// (column jf of H: crow[cptr[jf] .. cptr[jf+1])) in the residual; AND the
// window's convergence into conv.  One warp per shot.
__global__ void win_commit_kernel(const uint32_t *__restrict__ wcorr, int wvw, const int32_t *__restrict__ clocal,
                                  const int32_t *__restrict__ cfull, int ncommit, const int32_t *__restrict__ cptr,
                                  const int32_t *__restrict__ crow, uint32_t *__restrict__ corr, int wvf,
                                  uint32_t *__restrict__ resid, int wcf, const StatsDev *__restrict__ wstats,
                                  int32_t *__restrict__ conv, int64_t shots)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < shots; s += nwarp) {
        const uint32_t *wc = wcorr + s * wvw;
        for (int k = lane; k < ncommit; k += 32) {
            const int lc = __ldg(clocal + k);
            if (!((wc[lc >> 5] >> (lc & 31)) & 1u)) continue;
            const int jf = __ldg(cfull + k);
            atomicOr(corr + s * wvf + (jf >> 5), 1u << (jf & 31));
            for (int a = __ldg(cptr + jf), a1 = __ldg(cptr + jf + 1); a < a1; ++a) {
                const int i = __ldg(crow + a);
                atomicXor(resid + s * wcf + (i >> 5), 1u << (i & 31));
            }
        }
        if (lane == 0 && conv && !wstats[s].converged) conv[s] = 0;
    }
}

// Predicted observables O e^ of the committed correction; pobs must be zero.
// One warp per shot.
__global__ void win_obs_kernel(const uint32_t *__restrict__ corr, int wvf, int V, const int32_t *__restrict__ optr,
                               const int32_t *__restrict__ oidx, uint32_t *__restrict__ pobs, int wk, int64_t shots)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < shots; s += nwarp) {
        for (int w = lane; w < wvf; w += 32) {
            uint32_t x = corr[s * wvf + w];
            while (x) {
                const int b = __ffs(x) - 1;
                x &= x - 1u;
                const int j = w * 32 + b;
                if (j >= V) break;
                for (int q = __ldg(optr + j), qe = __ldg(optr + j + 1); q < qe; ++q) {
                    const int o = __ldg(oidx + q);
                    atomicXor(pobs + s * wk + (o >> 5), 1u << (o & 31));
                }
            }
        }
    }
}

__global__ void fill_i32_kernel(int32_t *__restrict__ out, int32_t v, int64_t n)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) out[q] = v;
}

}  // namespace relaybp
