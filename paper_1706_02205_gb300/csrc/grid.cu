#include <algorithm>
#include <cmath>
#include <vector>

#include "grid.cuh"

namespace kc {

Grid make_grid(int d, const double* lo, const double* hi, int64_t npts, double want, int64_t max_cells) {
    Grid g;
    g.dg = d < 3 ? d : 3;
    double ext[3] = {0, 0, 0};
    double vol = 1.0;
    int nz = 0;
    for (int t = 0; t < g.dg; ++t) {
        g.lo[t] = lo[t];
        ext[t] = hi[t] - lo[t];
        if (ext[t] > 0) {
            vol *= ext[t];
            nz++;
        }
    }
    double emax = 0;
    for (int t = 0; t < g.dg; ++t) emax = fmax(emax, ext[t]);
    if (!(emax > 0)) {
        g.c = 1.0;
        g.inv_c = 1.0;
        return g;
    }
    if (max_cells < 1) max_cells = 1;
    // smallest cell size allowed by the cell budget
    double cmin = nz > 0 ? pow(vol / (double)max_cells, 1.0 / nz) : emax;
    double c = want > 0 ? want : cmin;
    if (c < cmin) c = cmin;
    for (;;) {
        int64_t tot = 1;
        bool ok = true;
        for (int t = 0; t < g.dg; ++t) {
            double f = floor(ext[t] / c) + 1.0;
            if (f > 1e6) {
                ok = false;
                break;
            }
            g.n[t] = (int)f;
            tot *= g.n[t];
            if (tot > max_cells) {
                ok = false;
                break;
            }
        }
        if (ok) {
            g.ncells = tot;
            break;
        }
        c *= 1.25;
    }
    g.c = c;
    g.inv_c = 1.0 / c;
    return g;
}

__global__ void cell_keys_k(Grid g, const double* __restrict__ x, int d, const int32_t* __restrict__ ids, int64_t n,
                            uint64_t* __restrict__ key, int64_t* __restrict__ val, int* __restrict__ cnt) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) {
        int64_t id = ids ? ids[q] : q;
        int64_t c = cell_of(g, x + id * d);
        key[q] = (uint64_t)c;
        val[q] = id;
        atomicAdd(&cnt[c], 1);
    }
}
__global__ void ids_out_k(const int64_t* __restrict__ v, int64_t n, int32_t* __restrict__ out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) out[q] = (int32_t)v[q];
}

static int bits_of(int64_t v) {
    int b = 1;
    while (b < 63 && ((int64_t)1 << b) <= v) ++b;
    return b;
}

kc_status grid_build(const Grid& g, const double* x, int d, const int32_t* ids, int64_t n, int32_t* sorted,
                     int64_t* cell_start, Arena& A, cudaStream_t s) {
    uint64_t *k0, *k1;
    int64_t *v0, *v1;
    int* cnt;
    KC_TRY(A.get(&k0, n));
    KC_TRY(A.get(&k1, n));
    KC_TRY(A.get(&v0, n));
    KC_TRY(A.get(&v1, n));
    KC_TRY(A.get(&cnt, g.ncells));
    KC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * g.ncells, s));
    if (n > 0) ::kc::note_launch(), cell_keys_k<<<blocks_for(n, 256), 256, 0, s>>>(g, x, d, ids, n, k0, v0, cnt);
    KC_CUDA(cudaGetLastError());
    KC_TRY(exclusive_scan_i32_to_i64(cnt, cell_start, g.ncells, A, s));
    KC_TRY(radix_sort_u64_i64(k0, v0, k1, v1, n, bits_of(g.ncells), A, s));
    if (n > 0) ::kc::note_launch(), ids_out_k<<<blocks_for(n, 256), 256, 0, s>>>(v1, n, sorted);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

// per-block min/max over 3 axes, then a single-block fold
__global__ void bbox_k(const double* __restrict__ x, int64_t N, int d, double* __restrict__ part) {
    __shared__ double smin[3][256], smax[3][256];
    int dg = d < 3 ? d : 3;
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        for (int t = 0; t < dg; ++t) {
            double v = x[i * d + t];
            mn[t] = fmin(mn[t], v);
            mx[t] = fmax(mx[t], v);
        }
    for (int t = 0; t < 3; ++t) {
        smin[t][threadIdx.x] = mn[t];
        smax[t][threadIdx.x] = mx[t];
    }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int t = 0; t < 3; ++t) {
                smin[t][threadIdx.x] = fmin(smin[t][threadIdx.x], smin[t][threadIdx.x + o]);
                smax[t][threadIdx.x] = fmax(smax[t][threadIdx.x], smax[t][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int t = 0; t < 3; ++t) {
            part[blockIdx.x * 6 + t] = smin[t][0];
            part[blockIdx.x * 6 + 3 + t] = smax[t][0];
        }
}

kc_status bbox(const double* x, int64_t N, int d, double* lo, double* hi, Arena& A, cudaStream_t s) {
    const int nb = 128;
    double* part;
    KC_TRY(A.get(&part, nb * 6));
    ::kc::note_launch(), bbox_k<<<nb, 256, 0, s>>>(x, N, d, part);
    KC_CUDA(cudaGetLastError());
    double h[nb * 6];
    KC_CUDA(cudaMemcpyAsync(h, part, sizeof(h), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    for (int t = 0; t < 3; ++t) {
        lo[t] = INFINITY;
        hi[t] = -INFINITY;
        for (int b = 0; b < nb; ++b) {
            lo[t] = fmin(lo[t], h[b * 6 + t]);
            hi[t] = fmax(hi[t], h[b * 6 + 3 + t]);
        }
    }
    return KC_OK;
}

// per-block min and max of every coordinate
__global__ void bbox_all_k(const double* __restrict__ x, int64_t N, int d, double* __restrict__ part) {
    __shared__ double smin[8], smax[8];
    for (int t = 0; t < d; ++t) {
        double mn = INFINITY, mx = -INFINITY;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
            const double v = x[i * d + t];
            mn = fmin(mn, v);
            mx = fmax(mx, v);
        }
        for (int o = 16; o > 0; o >>= 1) {
            mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane_id() == 0) {
            smin[threadIdx.x >> 5] = mn;
            smax[threadIdx.x >> 5] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                mn = fmin(mn, smin[w]);
                mx = fmax(mx, smax[w]);
            }
            part[(blockIdx.x * d + t) * 2] = mn;
            part[(blockIdx.x * d + t) * 2 + 1] = mx;
        }
        __syncthreads();
    }
}

kc_status bbox_all(const double* x, int64_t N, int d, Origin* lo, double* E, Arena& A, cudaStream_t s) {
    if (d > MAXD) return fail(KC_EINVAL, "d must be <= 32");
    const int nb = 64;
    double* part;
    KC_TRY(A.get(&part, (size_t)nb * d * 2));
    ::kc::note_launch(), bbox_all_k<<<nb, 256, 0, s>>>(x, N, d, part);
    KC_CUDA(cudaGetLastError());
    double h[nb * MAXD * 2];
    KC_CUDA(cudaMemcpyAsync(h, part, sizeof(double) * nb * d * 2, cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    double e = 0.0;
    for (int t = 0; t < MAXD; ++t) lo->lo[t] = 0.0;
    for (int t = 0; t < d; ++t) {
        double mn = INFINITY, mx = -INFINITY;
        for (int b = 0; b < nb; ++b) {
            mn = fmin(mn, h[(b * d + t) * 2]);
            mx = fmax(mx, h[(b * d + t) * 2 + 1]);
        }
        lo->lo[t] = mn;
        e = fmax(e, mx - mn);
    }
    *E = e;
    return KC_OK;
}

// Per block: sum of x and of the products x_a x_b (a <= b, packed) over its
// points, a thread per pair.
__global__ void moments_k(const double* __restrict__ x, int64_t N, int d, double* __restrict__ part) {
    const int np = d * (d + 1) / 2;
    const int per = (int)((N + gridDim.x - 1) / gridDim.x);
    const int64_t q0 = (int64_t)blockIdx.x * per, q1 = min(N, q0 + per);
    for (int t = threadIdx.x; t < np + d; t += blockDim.x) {
        double s = 0.0;
        if (t < np) {
            int a = 0, r = t;  // pair (a, b) of the packed upper triangle
            while (r >= d - a) {
                r -= d - a;
                ++a;
            }
            const int b = a + r;
            for (int64_t q = q0; q < q1; ++q) s = fma(x[q * d + a], x[q * d + b], s);
        } else {
            const int a = t - np;
            for (int64_t q = q0; q < q1; ++q) s += x[q * d + a];
        }
        part[(int64_t)blockIdx.x * (np + d) + t] = s;
    }
}

struct Axes3 {
    double v[3][MAXD];
};
__global__ void project_k(const double* __restrict__ x, int64_t N, int d, Axes3 ax, double* __restrict__ out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N) return;
    for (int t = 0; t < 3; ++t) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s = fma(ax.v[t][k], x[q * d + k], s);
        out[q * 3 + t] = s;
    }
}

// Eigenvectors of the symmetric d x d matrix a (row-major, destroyed) by the
// cyclic Jacobi method: plane rotations that zero one off-diagonal entry at a
// time, accumulated in v (columns = eigenvectors), until the off-diagonal part
// is negligible; eigenvalues end on the diagonal of a.
static void jacobi_eigen(int d, double* a, double* v) {
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) v[i * d + j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                tot += a[i * d + j] * a[i * d + j];
                if (i != j) off += a[i * d + j] * a[i * d + j];
            }
        if (!(off > 1e-30 * tot)) break;
        for (int p = 0; p < d - 1; ++p)
            for (int q = p + 1; q < d; ++q) {
                const double apq = a[p * d + q];
                if (apq == 0.0) continue;
                const double theta = (a[q * d + q] - a[p * d + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < d; ++k) {  // columns p, q
                    const double akp = a[k * d + p], akq = a[k * d + q];
                    a[k * d + p] = c * akp - s * akq;
                    a[k * d + q] = s * akp + c * akq;
                }
                for (int k = 0; k < d; ++k) {  // rows p, q
                    const double apk = a[p * d + k], aqk = a[q * d + k];
                    a[p * d + k] = c * apk - s * aqk;
                    a[q * d + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < d; ++k) {
                    const double vkp = v[k * d + p], vkq = v[k * d + q];
                    v[k * d + p] = c * vkp - s * vkq;
                    v[k * d + q] = s * vkp + c * vkq;
                }
            }
    }
}

kc_status grid_coords(const double* x, int64_t N, int d, Arena& A, cudaStream_t s, const double** gx, int* gs) {
    if (d <= 3) {
        *gx = x;
        *gs = d;
        return KC_OK;
    }
    if (d > MAXD) return fail(KC_EINVAL, "d must be <= 32");
    const int np = d * (d + 1) / 2, nb = 152;
    double* part;
    KC_TRY(A.get(&part, (size_t)nb * (np + d)));
    ::kc::note_launch(), moments_k<<<nb, 256, 0, s>>>(x, N, d, part);
    KC_CUDA(cudaGetLastError());
    std::vector<double> h((size_t)nb * (np + d));
    KC_CUDA(cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    std::vector<double> m(np + d, 0.0), cov((size_t)d * d), vec((size_t)d * d);
    for (int b = 0; b < nb; ++b)
        for (int t = 0; t < np + d; ++t) m[t] += h[(size_t)b * (np + d) + t];
    for (int a = 0, t = 0; a < d; ++a)
        for (int b = a; b < d; ++b, ++t) {
            const double c = m[t] / (double)N - (m[np + a] / (double)N) * (m[np + b] / (double)N);
            cov[a * d + b] = cov[b * d + a] = c;
        }
    jacobi_eigen(d, cov.data(), vec.data());
    std::vector<int> idx(d);
    for (int i = 0; i < d; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int i, int j) { return cov[i * d + i] > cov[j * d + j]; });
    Axes3 ax;
    for (int t = 0; t < 3; ++t) {
        double nrm = 0.0;
        for (int k = 0; k < d; ++k) nrm += vec[k * d + idx[t]] * vec[k * d + idx[t]];
        nrm = std::sqrt(nrm);  // 1 up to rounding; renormalised so |v_t| <= 1 holds
        for (int k = 0; k < MAXD; ++k) ax.v[t][k] = k < d ? vec[k * d + idx[t]] / (nrm * (1.0 + 1e-14)) : 0.0;
    }
    double* out;
    KC_TRY(A.get(&out, (size_t)N * 3));
    ::kc::note_launch(), project_k<<<blocks_for(N, 256), 256, 0, s>>>(x, N, d, ax, out);
    KC_CUDA(cudaGetLastError());
    *gx = out;
    *gs = 3;
    return KC_OK;
}

}  // namespace kc
