// Mie scattering by a homogeneous sphere (Sec. 3.1: the radiance of a ray
// from a PIV particle, computed with the method of Bohren & Huffman), and the
// optics handle whose rays carry that radiance.
//
// The series: size parameter x = pi d n_medium / lambda, relative index m;
// a_n, b_n from the Riccati-Bessel functions psi_n(x) = x j_n(x),
// xi_n(x) = psi_n - i chi_n (upward recurrences) and the logarithmic
// derivative D_n(mx) (downward recurrence started above the last order);
// S1, S2 from the angular functions pi_n, tau_n of cos(theta); the series
// stops after x + 4 x^(1/3) + 2 terms.  FP64 throughout: the coefficients
// are one sequential recurrence (one thread), the angles are independent
// (one thread each).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "handles.cuh"

namespace pivbos {

struct cplx {
    double re, im;
};
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return cplx{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return cplx{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return cplx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cplx cscale(cplx a, double s) { return cplx{a.re * s, a.im * s}; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b)
{
    // Smith's division (no overflow for large |b|)
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, d = b.re + b.im * r;
        return cplx{(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    }
    const double r = b.re / b.im, d = b.re * r + b.im;
    return cplx{(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}

// a_n, b_n for n = 1..nstop (index n), and the efficiency sums.  One thread.
// D holds nmx + 1 entries of scratch.
__global__ void mie_coef_kernel(double x, double m_re, double m_im, int nstop, int nmx, cplx* __restrict__ D,
                                cplx* __restrict__ a, cplx* __restrict__ b, double* __restrict__ q)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const cplx m{m_re, m_im};
    const cplx z{m_re * x, m_im * x};
    D[nmx] = cplx{0.0, 0.0};
    for (int n = nmx; n >= 1; --n) {
        const cplx nz = cdiv(cplx{(double)n, 0.0}, z);
        D[n - 1] = csub(nz, cdiv(cplx{1.0, 0.0}, cadd(D[n], nz)));
    }
    double psi_m1 = cos(x), psi_0 = sin(x);   // psi_{-1}, psi_0
    double chi_m1 = -sin(x), chi_0 = cos(x);  // chi_{-1}, chi_0
    double qe = 0.0, qs = 0.0;
    for (int n = 1; n <= nstop; ++n) {
        const double psi_n = (2.0 * n - 1.0) / x * psi_0 - psi_m1;
        const double chi_n = (2.0 * n - 1.0) / x * chi_0 - chi_m1;
        const cplx xi_n{psi_n, -chi_n}, xi_p{psi_0, -chi_0};
        const cplx nx{(double)n / x, 0.0};
        const cplx ta = cadd(cdiv(D[n], m), nx);
        const cplx tb = cadd(cmul(m, D[n]), nx);
        const cplx an = cdiv(csub(cscale(ta, psi_n), cplx{psi_0, 0.0}), csub(cmul(ta, xi_n), xi_p));
        const cplx bn = cdiv(csub(cscale(tb, psi_n), cplx{psi_0, 0.0}), csub(cmul(tb, xi_n), xi_p));
        a[n] = an;
        b[n] = bn;
        qe += (2.0 * n + 1.0) * (an.re + bn.re);
        qs += (2.0 * n + 1.0) * (an.re * an.re + an.im * an.im + bn.re * bn.re + bn.im * bn.im);
        psi_m1 = psi_0;
        psi_0 = psi_n;
        chi_m1 = chi_0;
        chi_0 = chi_n;
    }
    q[0] = 2.0 / (x * x) * qe;
    q[1] = 2.0 / (x * x) * qs;
}

// |S1|^2, |S2|^2 at theta_i = pi i / (n_angles - 1); one thread per angle.
__global__ void mie_angles_kernel(int nstop, const cplx* __restrict__ a, const cplx* __restrict__ b, int n_angles,
                                  double* __restrict__ s12, double* __restrict__ q)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_angles) return;
    const double mu = cospi((double)i / (double)(n_angles - 1));
    double pi_prev = 0.0, pi_n = 1.0;   // pi_0, pi_1
    cplx S1{0.0, 0.0}, S2{0.0, 0.0};
    for (int n = 1; n <= nstop; ++n) {
        const double tau_n = n * mu * pi_n - (n + 1.0) * pi_prev;
        const double f = (2.0 * n + 1.0) / ((double)n * (n + 1.0));
        const cplx an = a[n], bn = b[n];
        S1 = cadd(S1, cscale(cadd(cscale(an, pi_n), cscale(bn, tau_n)), f));
        S2 = cadd(S2, cscale(cadd(cscale(an, tau_n), cscale(bn, pi_n)), f));
        const double pi_next = ((2.0 * n + 1.0) / n) * mu * pi_n - ((n + 1.0) / n) * pi_prev;
        pi_prev = pi_n;
        pi_n = pi_next;
    }
    s12[2 * i] = S1.re * S1.re + S1.im * S1.im;
    s12[2 * i + 1] = S2.re * S2.re + S2.im * S2.im;
    if (i == 0) q[2] = S1.re;
}

}  // namespace pivbos


extern "C" {

pivbos_status pivbos_mie(double diameter, double wavelength, double n_medium, double m_re, double m_im,
                         int n_angles, double* s12, double* q)
{
    using namespace pivbos;
    set_last_error("");
    if (!(diameter > 0.0 && wavelength > 0.0 && n_medium > 0.0 && m_re > 0.0 && m_im >= 0.0) ||
        !isfinite(diameter) || !isfinite(wavelength) || !isfinite(n_medium) || !isfinite(m_re) || !isfinite(m_im))
        return failf(PIVBOS_ERR_INVALID_ARG, "diameter, wavelength, indices");
    if (n_angles < 2 || n_angles > (1 << 20) || !s12) return failf(PIVBOS_ERR_INVALID_ARG, "n_angles or s12");
    const double x = M_PI * diameter * n_medium / wavelength;
    if (x > 20000.0) return failf(PIVBOS_ERR_UNSUPPORTED, "size parameter %.4g above 20000", x);
    const int nstop = (int)(x + 4.0 * cbrt(x) + 2.0);
    const int nmx = (int)fmax((double)nstop, x * hypot(m_re, m_im)) + 16;
    const size_t coef = (size_t)(nstop + 1) * sizeof(cplx);
    const size_t bytes = (size_t)(nmx + 1) * sizeof(cplx) + 2 * coef + (size_t)n_angles * 2 * sizeof(double) + 64;
    char* buf = nullptr;
    pivbos_status st = cuda_status(cudaMalloc((void**)&buf, bytes), "Mie scratch");
    if (st) return st;
    cplx* D = (cplx*)buf;
    cplx* a = (cplx*)(buf + (size_t)(nmx + 1) * sizeof(cplx));
    cplx* b = (cplx*)((char*)a + coef);
    double* ds12 = (double*)((char*)b + coef);
    double* dq = ds12 + (size_t)n_angles * 2;
    mie_coef_kernel<<<1, 32>>>(x, m_re, m_im, nstop, nmx, D, a, b, dq);
    mie_angles_kernel<<<(n_angles + 127) / 128, 128>>>(nstop, a, b, n_angles, ds12, dq);
    count_launches(2);
    cudaError_t e = cudaGetLastError();
    double hq[3] = {0.0, 0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpy(s12, ds12, (size_t)n_angles * 2 * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hq, dq, sizeof hq, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if ((st = cuda_status(e, "Mie kernels"))) return st;
    if (q) {
        q[0] = hq[0];
        q[1] = hq[1];
        q[2] = hq[2];
        q[3] = nstop;
    }
    return PIVBOS_OK;
}

pivbos_status pivbos_optics_radiance(const pivbos_optics* o, const double laser_dir[3], const double* polarisation,
                                     const double* s12, int n_angles, pivbos_optics** out)
{
    using namespace pivbos;
    set_last_error("");
    if (!o || !out || !laser_dir || !s12) return failf(PIVBOS_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (n_angles < 2 || n_angles > (1 << 20)) return failf(PIVBOS_ERR_INVALID_ARG, "n_angles %d", n_angles);
    const double ll = sqrt(laser_dir[0] * laser_dir[0] + laser_dir[1] * laser_dir[1] + laser_dir[2] * laser_dir[2]);
    if (!(ll > 0.0) || !isfinite(ll)) return failf(PIVBOS_ERR_INVALID_ARG, "laser direction");
    double L[3], P[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k) L[k] = laser_dir[k] / ll;
    if (polarisation) {
        const double pl = sqrt(polarisation[0] * polarisation[0] + polarisation[1] * polarisation[1] +
                               polarisation[2] * polarisation[2]);
        if (!(pl > 0.0) || !isfinite(pl)) return failf(PIVBOS_ERR_INVALID_ARG, "polarisation");
        for (int k = 0; k < 3; ++k) P[k] = polarisation[k] / pl;
        if (fabs(P[0] * L[0] + P[1] * L[1] + P[2] * L[2]) > 1e-6)
            return failf(PIVBOS_ERR_INVALID_ARG, "polarisation must be normal to the laser direction");
    }
    double mx = 0.0;
    for (int i = 0; i < 2 * n_angles; ++i) {
        if (!(s12[i] >= 0.0) || !isfinite(s12[i])) return failf(PIVBOS_ERR_INVALID_ARG, "table entry %d", i);
        mx = fmax(mx, s12[i]);
    }
    if (!(mx > 0.0)) return failf(PIVBOS_ERR_INVALID_ARG, "the table is zero");
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_status(cudaGetLastError(), "cudaGetDevice");
    if (o->device != dev) return failf(PIVBOS_ERR_INVALID_ARG, "optics handle belongs to device %d", o->device);
    float2* h = new (std::nothrow) float2[n_angles];
    if (!h) return failf(PIVBOS_ERR_OOM, "host allocation");
    for (int i = 0; i < n_angles; ++i) h[i] = make_float2((float)(s12[2 * i] / mx), (float)(s12[2 * i + 1] / mx));
    float2* d = nullptr;
    cudaError_t e = cudaMalloc((void**)&d, (size_t)n_angles * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemcpy(d, h, (size_t)n_angles * sizeof(float2), cudaMemcpyHostToDevice);
    delete[] h;
    if (e != cudaSuccess) {
        if (d) cudaFree(d);
        return cuda_status(e, "radiance table");
    }
    pivbos_optics* c = new (std::nothrow) pivbos_optics(*o);
    if (!c) {
        cudaFree(d);
        return failf(PIVBOS_ERR_OOM, "host allocation");
    }
    c->d.rad = d;
    c->d.rad_n = n_angles;
    c->d.rad_mode = polarisation ? 2 : 1;
    for (int k = 0; k < 3; ++k) {
        c->d.rad_L[k] = (float)L[k];
        c->d.rad_pol[k] = (float)P[k];
    }
    c->rad_owned = d;
    *out = c;
    return PIVBOS_OK;
}

}  // extern "C"
