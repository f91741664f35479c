// Joint Kalman-filter likelihood of a pulsar timing array with a stochastic
// GW background coupled by the Hellings-Downs correlation (include/argus_gwb.h).
//
// The state of all P pulsars, (rho_n, y_n, a_n), evolves together, and every
// TOA of every pulsar updates it, so the work per TOA is O(P^2) and the lanes
// are parameter vectors, not pulsars: one thread block per parameter vector
// with the 3P x 3P covariance in shared memory.  Per TOA:
//   1. transition coefficients over dt: each pulsar's OU red noise
//      (a_p, b_p, Q_p / sigma_p^2 by ou_coef) and the GW process's;
//   2. predict: F is block diagonal (3 x 3 per pulsar,
//      F_n = [[1, b_p, b_a], [0, a_p, 0], [0, 0, a_a]]), so each 3 x 3 block
//      of P becomes F_I P_IJ F_J^T + Q_IJ on its own.  P is symmetric and
//      only its upper triangle is stored: blocks I <= J are computed, the
//      diagonal blocks read symmetrically.  Q_IJ holds the intrinsic noise
//      (I = J) and h_a^2 G_IJ times the integrated-OU increment covariance of
//      the GW process in the (rho, a) slots;
//   3. innovate on rho_q of the TOA's pulsar q: c = P e_{3q}, S = c_{3q} + R,
//      e = r - m_{3q} (thread 0 forms 1/S once);
//   4. update: m += c e / S and, over the upper triangle only,
//      P_ij -= (c_i c_j) / S; accumulate -1/2 (ln 2 pi + ln S + e^2 / S).
// Steps 2-4 are spread over the block's threads with a barrier between them;
// a TOA at the same time as the previous one skips the predict (F = I, Q = 0).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/argus.h"
#include "../../include/argus_gwb.h"
#include "kf_internal.cuh"
#include "lib_internal.cuh"
#include "kf_math.cuh"
#include "kf_model.cuh"

namespace argus {
namespace {

constexpr double kLog2PiGwb = 1.8378770664093454836;
constexpr int kGwbThreads = 256;

struct GwbRec {     // one TOA of the merged, time-ordered stream (32 bytes)
    double dt;      // time since the previous TOA of any pulsar (0 for the first)
    double r;       // residual, s
    double s2;      // sigma_k^2
    int32_t q;      // pulsar
    int32_t pad;
};

struct GwbArgs {
    const GwbRec* rec;
    int64_t N;
    int32_t P;
    const double* p0;       // [P][3]
    const double* equad2;   // [P]
    const double* G;        // [P][P] Hellings-Downs
    const double* theta;    // [B][2 + 3P]
    int64_t B;
    double* loglik;         // [B]
};

__host__ __device__ inline size_t gwb_smem_doubles(int P) {
    const int n = 3 * P;
    // P, m, c, per-pulsar coefficients (5P), G, per-pulsar parameters (3P), GW coefficients + scalars
    return size_t(n) * n + 2 * n + 5 * P + size_t(P) * P + 3 * P + 16;
}

// dynamic shared memory of a block: the doubles, the (I, J) pairs of the
// upper 3x3 blocks (uint16) and the (i, j) pairs of the upper entries (uint8)
__host__ __device__ inline size_t gwb_smem_bytes(int P) {
    const size_t n = 3 * size_t(P);
    return gwb_smem_doubles(P) * sizeof(double) + size_t(P) * (P + 1) * sizeof(uint16_t) +
           n * (n + 1) * sizeof(uint8_t);
}

__global__ void __launch_bounds__(kGwbThreads) k_gwb_filter(GwbArgs a) {
    extern __shared__ __align__(16) double gsm[];
    const int P = a.P, n = 3 * P, D = 2 + 3 * P;
    double* Pm = gsm;                        // [n][n]
    double* m = Pm + size_t(n) * n;          // [n]
    double* c = m + n;                       // [n] column of the update
    double* co = c + n;                      // [P][5]: a_p, b_p, sigma^2 (q00, q01, q11)
    double* G = co + 5 * P;                  // [P][P]
    double* par = G + size_t(P) * P;         // [P][3]: sigma^2, gamma_p, EFAC^2
    double* gw = par + 3 * P;                // a_a, b_a, h_a^2 (q00, q01, q11), h_a^2, gamma_a, e, S, ok
    uint16_t* pairs = reinterpret_cast<uint16_t*>(gw + 16);   // upper 3x3 blocks (I, J)
    const int nb = P * (P + 1) / 2;
    uint8_t* ent = reinterpret_cast<uint8_t*>(pairs + 2 * nb);   // upper entries (i, j), i <= j
    const int ne = n * (n + 1) / 2;
    const int tid = threadIdx.x;
    for (int i = tid; i < P * P; i += blockDim.x) G[i] = a.G[i];
    if (tid == 0) {
        int k = 0;
        for (int I = 0; I < P; ++I)
            for (int J = I; J < P; ++J) { pairs[2 * k] = uint16_t(I); pairs[2 * k + 1] = uint16_t(J); ++k; }
        k = 0;
        for (int i = 0; i < n; ++i)
            for (int j = i; j < n; ++j) { ent[2 * k] = uint8_t(i); ent[2 * k + 1] = uint8_t(j); ++k; }
    }
    for (int64_t b = blockIdx.x; b < a.B; b += gridDim.x) {
        const double* th = a.theta + b * D;
        __syncthreads();
        if (tid == 0) {
            bool ok = true;
            for (int j = 0; j < D; ++j) ok = ok && isfinite(th[j]);
            for (int p = 0; p < P; ++p) ok = ok && th[2 + 3 * p + 2] > 0.0;
            gw[5] = exp10(2.0 * th[0]);
            gw[6] = exp10(th[1]);
            gw[9] = ok ? 1.0 : 0.0;
        }
        for (int p = tid; p < P; p += blockDim.x) {
            par[3 * p] = exp10(2.0 * th[2 + 3 * p]);
            par[3 * p + 1] = exp10(th[2 + 3 * p + 1]);
            const double ef = th[2 + 3 * p + 2];
            par[3 * p + 2] = ef * ef;
        }
        __syncthreads();
        if (gw[9] == 0.0) {
            if (tid == 0) a.loglik[b] = -INFINITY;
            continue;
        }
        // prior at the array's earliest TOA
        const double ha2 = gw[5], ga = gw[6];
        for (int i = tid; i < n * n; i += blockDim.x) {
            const int r = i / n, col = i - r * n;
            const int I = r / 3, J = col / 3, u = r - 3 * I, v = col - 3 * J;
            double x = 0.0;
            if (u == 2 && v == 2) x = ha2 * G[I * P + J] / (2.0 * ga);
            else if (I == J && u < 2 && v < 2) x = a.p0[3 * I + u + v];
            Pm[i] = x;
        }
        for (int i = tid; i < n; i += blockDim.x) m[i] = 0.0;
        double quad = 0.0;
        LogProd lp;
        __syncthreads();
        for (int64_t k = 0; k < a.N; ++k) {
            const GwbRec rk = a.rec[k];
            const double dt = rk.dt;
            if (dt > 0.0) {
                // 1. transition coefficients
                const double h2 = 0.5 * dt * dt, h3 = dt * dt * dt / 3.0;
                for (int p = tid; p <= P; p += blockDim.x) {
                    OuCoef oc;
                    if (p < P) {
                        ou_coef<false>(par[3 * p + 1] * dt, dt, h2, h3, 0.0, oc);
                        const double s2 = par[3 * p];
                        co[5 * p] = oc.a; co[5 * p + 1] = oc.b;
                        co[5 * p + 2] = s2 * oc.c00; co[5 * p + 3] = s2 * oc.c01; co[5 * p + 4] = s2 * oc.c11;
                    } else {
                        ou_coef<false>(ga * dt, dt, h2, h3, 0.0, oc);
                        gw[0] = oc.a; gw[1] = oc.b;
                        gw[2] = ha2 * oc.c00; gw[3] = ha2 * oc.c01; gw[4] = ha2 * oc.c11;
                    }
                }
                __syncthreads();
                // 2. predict the mean (one thread per pulsar) and each upper block
                const double aa = gw[0], ba = gw[1], qa00 = gw[2], qa01 = gw[3], qa11 = gw[4];
                for (int p = tid; p < P; p += blockDim.x) {
                    double* mp = m + 3 * p;
                    mp[0] = fma(co[5 * p + 1], mp[1], fma(ba, mp[2], mp[0]));
                    mp[1] *= co[5 * p];
                    mp[2] *= aa;
                }
                for (int q = tid; q < nb; q += blockDim.x) {
                    const int I = pairs[2 * q], J = pairs[2 * q + 1];
                    const double apI = co[5 * I], bpI = co[5 * I + 1];
                    const double apJ = co[5 * J], bpJ = co[5 * J + 1];
                    double X[3][3];
                    for (int u = 0; u < 3; ++u)
                        for (int v = 0; v < 3; ++v)
                            X[u][v] = (I < J || u <= v) ? Pm[(3 * I + u) * n + 3 * J + v]
                                                        : Pm[(3 * I + v) * n + 3 * J + u];
                    double Y[3][3];   // F_I X
                    for (int v = 0; v < 3; ++v) {
                        Y[0][v] = fma(bpI, X[1][v], fma(ba, X[2][v], X[0][v]));
                        Y[1][v] = apI * X[1][v];
                        Y[2][v] = aa * X[2][v];
                    }
                    double Z[3][3];   // (F_I X) F_J^T
                    for (int u = 0; u < 3; ++u) {
                        Z[u][0] = fma(bpJ, Y[u][1], fma(ba, Y[u][2], Y[u][0]));
                        Z[u][1] = apJ * Y[u][1];
                        Z[u][2] = aa * Y[u][2];
                    }
                    const double g = G[I * P + J];
                    Z[0][0] = fma(g, qa00, Z[0][0]);
                    Z[0][2] = fma(g, qa01, Z[0][2]);
                    Z[2][0] = fma(g, qa01, Z[2][0]);
                    Z[2][2] = fma(g, qa11, Z[2][2]);
                    if (I == J) {
                        Z[0][0] += co[5 * I + 2];
                        Z[0][1] += co[5 * I + 3];
                        Z[1][0] += co[5 * I + 3];
                        Z[1][1] += co[5 * I + 4];
                    }
                    for (int u = 0; u < 3; ++u)
                        for (int v = 0; v < 3; ++v)
                            if (I < J || u <= v) Pm[(3 * I + u) * n + 3 * J + v] = Z[u][v];
                }
                __syncthreads();
            }
            // 3. innovate on rho of pulsar q
            const int i0 = 3 * rk.q;
            for (int i = tid; i < n; i += blockDim.x) c[i] = Pm[min(i, i0) * n + max(i, i0)];
            if (tid == 0) {
                const double R = fma(par[3 * rk.q + 2], rk.s2, a.equad2[rk.q]);
                const double e = rk.r - m[i0];
                const double S = Pm[i0 * n + i0] + R;
                const double rS = rcp_nr(S);
                gw[7] = rS;
                gw[8] = e * rS;
                quad = fma(e, gw[8], quad);
                lp.add(S);
            }
            __syncthreads();
            // 4. update (upper triangle)
            const double rS = gw[7], g = gw[8];
            for (int q = tid; q < ne; q += blockDim.x) {
                const int r = ent[2 * q], col = ent[2 * q + 1];
                Pm[r * n + col] = fma(-(c[r] * c[col]), rS, Pm[r * n + col]);
            }
            for (int i = tid; i < n; i += blockDim.x) m[i] = fma(c[i], g, m[i]);
            __syncthreads();
        }
        if (tid == 0) {
            double ll = (a.N == 0) ? 0.0 : -0.5 * (double(a.N) * kLog2PiGwb + lp.value() + quad);
            if (lp.bad || !isfinite(ll)) ll = -INFINITY;
            a.loglik[b] = ll;
        }
    }
}

}  // namespace
}  // namespace argus

using namespace argus;

struct argus_gwb {
    int device = 0;
    int n_sm = 0;
    int P = 0;
    int64_t N = 0;
    GwbRec* d_rec = nullptr;
    double* d_p0 = nullptr;
    double* d_equad2 = nullptr;
    double* d_G = nullptr;
    double* d_stage = nullptr;
    size_t cap_stage = 0;
};

namespace {

int gwb_fail(int st, const std::string& msg) { return record_error(st, msg.c_str()); }

int gwb_cuda(cudaError_t e, const char* what) {
    return record_error(e == cudaErrorMemoryAllocation ? ARGUS_ERR_OOM : ARGUS_ERR_CUDA,
                        (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

// Hellings-Downs matrix: G_nm = 3/2 x ln x - x/4 + 1/2, x = (1 - c_n.c_m)/2; G_nn = 1.
std::vector<double> hellings_downs(const argus_pulsar* psrs, int P) {
    std::vector<double> G(size_t(P) * P);
    for (int a = 0; a < P; ++a)
        for (int b = 0; b < P; ++b) {
            if (a == b) { G[size_t(a) * P + b] = 1.0; continue; }
            double cth = 0.0;
            for (int i = 0; i < 3; ++i) cth += psrs[a].pos[i] * psrs[b].pos[i];
            cth = std::min(1.0, std::max(-1.0, cth));
            const double x = 0.5 * (1.0 - cth);
            G[size_t(a) * P + b] = (x > 0.0 ? 1.5 * x * std::log(x) : 0.0) - 0.25 * x + 0.5;
        }
    return G;
}

bool gwb_is_device_ptr(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

argus_status argus_gwb_create(const argus_pulsar* psrs, int32_t n_pulsars, int32_t device,
                              argus_gwb** out) {
    if (!out) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "out is NULL"));
    if (!psrs || n_pulsars < 1) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "need at least one pulsar"));
    if (n_pulsars > kGwbMaxPulsars)
        return argus_status(gwb_fail(ARGUS_ERR_UNSUPPORTED, "the joint filter holds at most 48 pulsars"));
    if (device < 0) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "device must be >= 0"));
    int64_t total = 0;
    if (int st = validate_pulsars(psrs, n_pulsars, &total)) return argus_status(st);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return argus_status(gwb_cuda(e, "cudaGetDeviceCount"));
    if (device >= ndev) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "no such device"));
    cudaDeviceProp prop{};
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess)
        return argus_status(gwb_cuda(e, "cudaGetDeviceProperties"));
    if (prop.major != 10 || prop.minor != 3)
        return argus_status(gwb_fail(ARGUS_ERR_UNSUPPORTED, std::string("built for sm_103a, device is ") + prop.name));
    // merged TOA stream, time order; ties keep (pulsar, TOA) order
    std::vector<int32_t> psr_of;
    std::vector<int64_t> loc;
    psr_of.reserve(size_t(total));
    loc.reserve(size_t(total));
    for (int p = 0; p < n_pulsars; ++p)
        for (int64_t k = 0; k < psrs[p].n_toa; ++k) { psr_of.push_back(p); loc.push_back(k); }
    std::vector<int64_t> order(static_cast<size_t>(total));
    std::iota(order.begin(), order.end(), int64_t(0));
    auto tof = [&](int64_t g) { return psrs[psr_of[g]].t[loc[g]]; };
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return tof(x) < tof(y); });
    std::vector<GwbRec> rec(size_t(std::max<int64_t>(total, 1)));
    double t_prev = total ? tof(order[0]) : 0.0;
    for (int64_t j = 0; j < total; ++j) {
        const int64_t g = order[j];
        const argus_pulsar& ps = psrs[psr_of[g]];
        const double t = ps.t[loc[g]];
        rec[j] = GwbRec{t - t_prev, ps.r[loc[g]], ps.sigma[loc[g]] * ps.sigma[loc[g]], psr_of[g], 0};
        t_prev = t;
    }
    std::vector<double> p0(size_t(3) * n_pulsars), eq2(n_pulsars);
    for (int p = 0; p < n_pulsars; ++p) {
        for (int i = 0; i < 3; ++i) p0[3 * p + i] = psrs[p].p0[i];
        eq2[p] = psrs[p].equad * psrs[p].equad;
    }
    const std::vector<double> G = hellings_downs(psrs, n_pulsars);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    argus_gwb* h = new argus_gwb();
    h->device = device;
    h->n_sm = prop.multiProcessorCount;
    h->P = n_pulsars;
    h->N = total;
    auto bail = [&](cudaError_t err, const char* what) {
        argus_gwb_destroy(h);
        if (prev >= 0) cudaSetDevice(prev);
        return argus_status(gwb_cuda(err, what));
    };
    if ((e = cudaMalloc(&h->d_rec, sizeof(GwbRec) * rec.size())) != cudaSuccess) return bail(e, "cudaMalloc(records)");
    if ((e = cudaMalloc(&h->d_p0, sizeof(double) * p0.size())) != cudaSuccess) return bail(e, "cudaMalloc(p0)");
    if ((e = cudaMalloc(&h->d_equad2, sizeof(double) * eq2.size())) != cudaSuccess) return bail(e, "cudaMalloc(equad)");
    if ((e = cudaMalloc(&h->d_G, sizeof(double) * G.size())) != cudaSuccess) return bail(e, "cudaMalloc(G)");
    if ((e = cudaMemcpy(h->d_rec, rec.data(), sizeof(GwbRec) * rec.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->d_p0, p0.data(), sizeof(double) * p0.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->d_equad2, eq2.data(), sizeof(double) * eq2.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->d_G, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "cudaMemcpy");
    // the kernel's dynamic shared memory limit, set for the largest array any
    // handle may hold (a per-function setting shared by all handles)
    const size_t smem_max = gwb_smem_bytes(kGwbMaxPulsars);
    if ((e = cudaFuncSetAttribute(k_gwb_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_max))) !=
        cudaSuccess)
        return bail(e, "cudaFuncSetAttribute");
    if (prev >= 0) cudaSetDevice(prev);
    *out = h;
    return ARGUS_OK;
}

void argus_gwb_destroy(argus_gwb* h) {
    if (!h) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    cudaFree(h->d_rec);
    cudaFree(h->d_p0);
    cudaFree(h->d_equad2);
    cudaFree(h->d_G);
    cudaFree(h->d_stage);
    if (prev >= 0) cudaSetDevice(prev);
    delete h;
}

int32_t argus_gwb_dim(const argus_gwb* h) { return h ? 2 + 3 * h->P : -1; }

argus_status argus_gwb_loglik(argus_gwb* h, const double* theta, int64_t B, double* loglik,
                              void* stream) {
    if (!h) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "handle is NULL"));
    if (B < 0) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "B must be >= 0"));
    if (B == 0) return ARGUS_OK;
    if (!theta || !loglik) return argus_status(gwb_fail(ARGUS_ERR_INVALID_ARG, "theta or loglik is NULL"));
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int D = 2 + 3 * h->P;
    const bool dev_in = gwb_is_device_ptr(theta), dev_out = gwb_is_device_ptr(loglik);
    const double* th_d = theta;
    double* ll_d = loglik;
    cudaError_t e = cudaSuccess;
    argus_status st = ARGUS_OK;
    if (!dev_in || !dev_out) {
        const size_t need = size_t(B) * (D + 1);
        if (need > h->cap_stage) {
            cudaFree(h->d_stage);
            h->d_stage = nullptr;
            h->cap_stage = 0;
            if ((e = cudaMalloc(&h->d_stage, need * sizeof(double))) != cudaSuccess) {
                st = argus_status(gwb_cuda(e, "cudaMalloc(stage)"));
                goto done;
            }
            h->cap_stage = need;
        }
        if (!dev_in) {
            if ((e = cudaMemcpyAsync(h->d_stage, theta, sizeof(double) * B * D, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess) {
                st = argus_status(gwb_cuda(e, "cudaMemcpyAsync(theta)"));
                goto done;
            }
            th_d = h->d_stage;
        }
        if (!dev_out) ll_d = h->d_stage + size_t(B) * D;
    }
    {
        GwbArgs a{h->d_rec, h->N, h->P, h->d_p0, h->d_equad2, h->d_G, th_d, B, ll_d};
        const size_t smem = gwb_smem_bytes(h->P);
        const int grid = int(std::min<int64_t>(B, int64_t(h->n_sm) * 8));
        k_gwb_filter<<<grid, kGwbThreads, smem, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            st = argus_status(gwb_cuda(e, "k_gwb_filter"));
            goto done;
        }
        if (!dev_out) {
            if ((e = cudaMemcpyAsync(loglik, ll_d, sizeof(double) * B, cudaMemcpyDeviceToHost, s)) != cudaSuccess) {
                st = argus_status(gwb_cuda(e, "cudaMemcpyAsync(loglik)"));
                goto done;
            }
        }
        if (!dev_in || !dev_out) {
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) st = argus_status(gwb_cuda(e, "cudaStreamSynchronize"));
        }
    }
done:
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}

}  // extern "C"
