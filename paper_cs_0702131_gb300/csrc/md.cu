// Time integration for the paper's verification runs (§3: energy and
// momentum conservation, independence of the mesh): the velocity-Verlet
// scheme around the per-step hot path (binning and forces).
//
//   v += (dt / 2) F(t) / m;  x += dt v;  bin;  F(t + dt);  v += (dt / 2) F(t + dt) / m
//
// Kernels: md_kick (FP32 or FP64 forces), md_drift, md_kinetic (FP64 kinetic
// energy and momentum, block sums and one atomic per block and value).
#include <math.h>

#include <algorithm>

#include "aica_internal.cuh"

namespace aica {
namespace {

struct MdArgs {
    int64_t n;
    const int32_t *species;
    double inv_m[kMaxSpecies], m[kMaxSpecies];
};

template <class T>
__global__ void __launch_bounds__(256) md_kick(MdArgs a, const T *force, double *vel, double half_dt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * a.n) return;
    const int s = a.species[i / 3] & (kMaxSpecies - 1);
    vel[i] = fma(half_dt * a.inv_m[s], (double)force[i], vel[i]);
}

__global__ void __launch_bounds__(256) md_drift(int64_t n3, const double *vel, double *pos, double dt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3) pos[i] = fma(dt, vel[i], pos[i]);
}

// out[0] += sum m v^2 / 2, out[1..3] += sum m v
__global__ void __launch_bounds__(256) md_kinetic(MdArgs a, const double *vel, double *out) {
    __shared__ double sh[4][8];
    double k = 0, px = 0, py = 0, pz = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const double m = a.m[a.species[i] & (kMaxSpecies - 1)];
        const double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
        k += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        px += m * vx;
        py += m * vy;
        pz += m * vz;
    }
    double v[4] = {k, px, py, pz};
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j = 0; j < 4; ++j) {
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
        if (lane == 0) sh[j][w] = v[j];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[threadIdx.x][q];
        atomicAdd(out + threadIdx.x, t);
    }
}

aica_status fill_md(const aica_lj *lj, const double *mass, const int32_t *species, int64_t n, MdArgs &a) {
    if (!lj || !mass || lj->n_species < 1 || lj->n_species > kMaxSpecies) {
        set_error("aica_verlet_step: need masses for 1..%d species", kMaxSpecies);
        return AICA_ERR_INVALID_ARG;
    }
    a.n = n;
    a.species = species;
    for (int s = 0; s < kMaxSpecies; ++s) a.m[s] = a.inv_m[s] = 0.0;
    for (int s = 0; s < lj->n_species; ++s) {
        if (!(mass[s] > 0) || !isfinite(mass[s])) {
            set_error("aica_verlet_step: mass of species %d must be positive", s);
            return AICA_ERR_INVALID_ARG;
        }
        a.m[s] = mass[s];
        a.inv_m[s] = 1.0 / mass[s];
    }
    return AICA_OK;
}

}  // namespace
}  // namespace aica

using namespace aica;

extern "C" aica_status aica_verlet_step(aica_mesh *m, const aica_lj *lj, aica_precision prec, const double *mass,
                                        double dt, int64_t n, const int32_t *species, double *pos, double *vel,
                                        void *force, double *ev_out, double *kin_out, void *stream) {
    AICA_RANGE("aica_verlet_step");
    if (!m || !pos || !vel || !force || !species || n < 1) {
        set_error("aica_verlet_step: NULL argument or no molecules");
        return AICA_ERR_INVALID_ARG;
    }
    if (prec != AICA_FP32 && prec != AICA_FP64) { set_error("aica_verlet_step: bad precision"); return AICA_ERR_INVALID_ARG; }
    if (!(dt > 0) || !isfinite(dt)) { set_error("aica_verlet_step: dt must be positive"); return AICA_ERR_INVALID_ARG; }
    if (!m->built) { set_error("aica_verlet_step: build the lists first"); return AICA_ERR_NOT_BUILT; }
    if (m->n_owned >= 0) { set_error("aica_verlet_step: not available in portion mode (halo molecules)"); return AICA_ERR_INVALID_ARG; }
    MdArgs a{};
    aica_status s = fill_md(lj, mass, species, n, a);
    if (s != AICA_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned g3 = (unsigned)((3 * n + 255) / 256);
    const bool f64 = prec == AICA_FP64;
    if (f64) md_kick<double><<<g3, 256, 0, st>>>(a, (const double *)force, vel, 0.5 * dt);
    else md_kick<float><<<g3, 256, 0, st>>>(a, (const float *)force, vel, 0.5 * dt);
    md_drift<<<g3, 256, 0, st>>>(3 * n, vel, pos, dt);
    AICA_CUDA(cudaGetLastError());
    s = aica_bin_molecules(m, pos, species, n, nullptr, nullptr, nullptr, stream);
    if (s != AICA_OK) return s;
    const int64_t lb = m->launches;
    s = aica_forces(m, lj, prec, force, ev_out, nullptr, stream);
    if (s != AICA_OK) return s;
    if (f64) md_kick<double><<<g3, 256, 0, st>>>(a, (const double *)force, vel, 0.5 * dt);
    else md_kick<float><<<g3, 256, 0, st>>>(a, (const float *)force, vel, 0.5 * dt);
    int launches = 3;
    if (kin_out) {
        AICA_CUDA(cudaMemsetAsync(kin_out, 0, 4 * sizeof(double), st));
        md_kinetic<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 4), 256, 0, st>>>(a, vel, kin_out);
        ++launches;
    }
    AICA_CUDA(cudaGetLastError());
    m->launches += lb + launches;
    return AICA_OK;
}

extern "C" aica_status aica_kinetic(const double *mass, int32_t n_species, const int32_t *species, int64_t n,
                                    const double *vel, double *kin_out, void *stream) {
    if (!mass || !species || !vel || !kin_out || n < 0) { set_error("aica_kinetic: NULL argument"); return AICA_ERR_INVALID_ARG; }
    aica_lj lj{};
    lj.n_species = n_species;
    MdArgs a{};
    aica_status s = fill_md(&lj, mass, species, n, a);
    if (s != AICA_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    AICA_CUDA(cudaMemsetAsync(kin_out, 0, 4 * sizeof(double), st));
    if (n > 0) md_kinetic<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 4), 256, 0, st>>>(a, vel, kin_out);
    AICA_CUDA(cudaGetLastError());
    return AICA_OK;
}
