// FP64 canonical-embedding encoder (Appendix A.1.2 of the paper).
//
// Slot j of a real polynomial m is m(zeta^(5^j)), zeta = exp(i pi / N).  For
// real slot values z the preimage is m_i = (2/N) Re(sum_j z_j w^(i e_j)),
// w = exp(-2 pi i / 2N), e_j = 5^j mod 2N.  Every e_j is odd, e_j = 2 u_j + 1,
// so the sum is w^i * G[i] with G the N-point DFT of the vector holding z_j
// at position u_j.  G is computed by a radix-2 Stockham transform (one launch
// per stage over the whole batch), then twisted and scaled.  This is the only
// floating-point code on the device; it runs when a database is uploaded.
#include "internal.h"

namespace tetris {

namespace {

__global__ void zero_kernel(double2 *v, size_t total) {
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < total; it += (size_t)gridDim.x * blockDim.x)
        v[it] = make_double2(0.0, 0.0);
}

__global__ void scatter2_kernel(const double *slots, double2 *v, const int *u_of_j, int batch, int log_n) {
    const size_t n = (size_t)1 << log_n, half = n / 2;
    const size_t total = half * batch;
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < total; it += (size_t)gridDim.x * blockDim.x) {
        const size_t b = it / half, j = it % half;
        v[b * n + u_of_j[j]] = make_double2(slots[it], 0.0);
    }
}

// Stockham radix-2 DIF stage: sub-transform length len, stride s (len * s = N)
__global__ void stockham_kernel(const double2 *x, double2 *y, const double2 *tw, int batch, int log_n, int len, int s) {
    const size_t n = (size_t)1 << log_n, half = n / 2;
    const size_t total = half * batch;
    const int m = len / 2;
    const int tstep = (int)(n / len);
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < total; it += (size_t)gridDim.x * blockDim.x) {
        const size_t b = it / half, k = it % half;
        const int p = (int)(k / s), qq = (int)(k % s);
        const double2 *xb = x + b * n;
        double2 *yb = y + b * n;
        const double2 a = xb[qq + (size_t)s * p], c = xb[qq + (size_t)s * (p + m)];
        const double2 w = tw[(size_t)p * tstep];
        const double2 d = make_double2(__dsub_rn(a.x, c.x), __dsub_rn(a.y, c.y));
        yb[qq + (size_t)s * (2 * p)] = make_double2(__dadd_rn(a.x, c.x), __dadd_rn(a.y, c.y));
        yb[qq + (size_t)s * (2 * p + 1)] = make_double2(__dsub_rn(__dmul_rn(d.x, w.x), __dmul_rn(d.y, w.y)),
                                                          __dadd_rn(__dmul_rn(d.x, w.y), __dmul_rn(d.y, w.x)));
    }
}

__global__ void twist_kernel(const double2 *g, const double2 *twist, double *m, int batch, int log_n) {
    const size_t n = (size_t)1 << log_n;
    const size_t total = n * batch;
    const double f = 2.0 / (double)n;
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < total; it += (size_t)gridDim.x * blockDim.x) {
        const size_t i = it % n;
        const double2 a = g[it], w = twist[i];
        m[it] = __dmul_rn(f, __dsub_rn(__dmul_rn(a.x, w.x), __dmul_rn(a.y, w.y)));
    }
}

__global__ void db_slots_kernel(const uint8_t *vals, uint64_t records, int attrs, int blocks, int log_n, double *slots) {
    const size_t half = (size_t)1 << (log_n - 1);
    const size_t total = half * attrs * blocks;
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < total; it += (size_t)gridDim.x * blockDim.x) {
        const size_t i = it % half;
        const size_t a = (it / half) % attrs;
        const size_t b = it / (half * attrs);
        const uint64_t r = b * half + i;
        double z = 0.0;
        if (r < records) {
            const double v = (double)vals[r * attrs + a];
            z = __ddiv_rn(__ddiv_rn(__dsub_rn(v, 127.5), 127.5), (double)attrs);
        }
        slots[it] = z;
    }
}

__global__ void round_kernel(const double *m, int64_t *out, size_t count, double scale) {
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < count; it += (size_t)gridDim.x * blockDim.x)
        out[it] = (int64_t)floor(__dadd_rn(__dmul_rn(scale, m[it]), 0.5));
}

int blocks_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, (size_t)sm_count() * 16); }

}  // namespace

// twid_dev layout: [N/2] double2 DFT twiddles exp(-2 pi i k / N), then [N] double2
// twist exp(-pi i k / N), then [N/2] int u_j (as the bytes of an int array).
void encode_real_batch(const double *slots, double *m, int batch, int log_n, const double *twid_dev, double *work,
                       cudaStream_t s) {
    const size_t n = (size_t)1 << log_n;
    // every buffer is read and written as double2: 16-byte alignment, checked here
    TREQUIRE(((uintptr_t)twid_dev & 15) == 0 && ((uintptr_t)work & 15) == 0, -1,
             "encoder: twiddle table or work buffer not 16-byte aligned");
    const double2 *tw = reinterpret_cast<const double2 *>(twid_dev);
    const double2 *twist = tw + n / 2;
    const int *u_of_j = reinterpret_cast<const int *>(twist + n);
    double2 *x = reinterpret_cast<double2 *>(work);
    double2 *y = x + n * batch;
    zero_kernel<<<blocks_for(n * batch), 256, 0, s>>>(x, n * batch);
    scatter2_kernel<<<blocks_for(n / 2 * batch), 256, 0, s>>>(slots, x, u_of_j, batch, log_n);
    int len = (int)n, st = 1;
    while (len > 1) {
        stockham_kernel<<<blocks_for(n / 2 * batch), 256, 0, s>>>(x, y, tw, batch, log_n, len, st);
        std::swap(x, y);
        len /= 2;
        st *= 2;
    }
    twist_kernel<<<blocks_for(n * batch), 256, 0, s>>>(x, twist, m, batch, log_n);
}

void db_slots(const uint8_t *vals, uint64_t records, int attrs, int blocks, int log_n, double *slots, cudaStream_t s) {
    const size_t total = ((size_t)1 << (log_n - 1)) * attrs * blocks;
    db_slots_kernel<<<blocks_for(total), 256, 0, s>>>(vals, records, attrs, blocks, log_n, slots);
}

void round_scale(const double *m, int64_t *out, size_t count, double scale, cudaStream_t s) {
    round_kernel<<<blocks_for(count), 256, 0, s>>>(m, out, count, scale);
}

}  // namespace tetris
