// ntt_fourier.cu -- fused products with the FourierREDC twiddle multiply.
//
// The single-CTA product kernels of ntt.cu (N <= 2^14), instantiated with
// Alg. 3 (FourierREDC) in place of Alg. 2 (REDC) for every twiddle, scaling
// and pointwise multiply.  Alg. 3 trades the multiply by P' and by P for two
// multiplies by c 2^n = P - 1 and sign-mask corrections; it needs a Fourier
// prime P = c 2^n + 1 with 2n >= 32 and, for its 31-bit sign tests,
// P < 2^30.  Both reductions return a b R^-1 mod P, so the twiddle tables
// are shared and the results equal polymul_many's bit for bit; this entry
// point exists to compare the two reductions on the same kernels.
#include "ntt_internal.cuh"
#include "ntt_kernels.cuh"

namespace mont {
namespace {

int dispatch_fourier(int log2n, const PolyArgs &A, cudaStream_t s)
{
    switch (log2n) {
#define X(L) \
    case L: return launch_polymul_smem<L, RedAlg3>(A, s);
        X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14)
#undef X
    default: return MONT_EUNSUPPORTED;
    }
}

}  // namespace
}  // namespace mont

extern "C" int polymul_many_fourier(uint32_t p, const uint32_t *a, size_t la, const uint32_t *b, size_t lb,
                                    uint32_t *c, size_t count, cudaStream_t stream)
{
    if (count == 0) return MONT_OK;
    ntt_plan plan;
    int log2n = 0;
    const int rc = mont::polymul_prepare(p, a, la, b, lb, c, count, &plan, &log2n);
    if (rc != MONT_OK) return rc;
    if (p >= (1u << 30) || 2 * mont::two_adicity(p) < 32) return MONT_ERANGE;
    if (log2n > mont::kMaxSmemLog2N) return MONT_EUNSUPPORTED;
    mont::PolyArgs A;
    A.a = a;
    A.b = b;
    A.c = c;
    A.la = la;
    A.lb = lb;
    A.lc = la + lb - 1;
    A.count = count;
    A.tw = plan.table->fwd;
    A.itw = plan.table->inv;
    A.p = p;
    A.pp = plan.p_prime;
    A.k_scale = plan.k_scale;
    return mont::dispatch_fourier(log2n, A, stream);
}
