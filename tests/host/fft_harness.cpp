// CPU check of the shared-memory FFT groups of csrc/fft.cuh: the same
// dif_group / dit_group code, driven sequentially on the host, against an
// explicit O(N^2) DFT in double precision, for interleaved and split
// (re/im planes) batches of three sequences.  Prints the worst relative error
// per length and transform kind; exit status 1 when any exceeds 1e-5.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_2505_00387_gb300/csrc/fft.cuh"

using namespace aahrt;

static std::vector<float2> twiddles(int L) {
    const int N = 1 << L;
    std::vector<float2> tw(N);
    for (int m = 0; m < N; ++m) {
        const double a = -2.0 * M_PI * m / N;
        tw[m] = make_float2((float)cos(a), (float)sin(a));
    }
    return tw;
}

template <bool DIF, bool INV, class Batch>
static void run(const Batch &b, int nb, int L, const float2 *tw) {
    host_fft<DIF, INV>(b, nb, L, tw);
}

int main() {
    srand(1234);
    double worst_all = 0.0;
    const int NB = 3;
    for (int L = 1; L <= 13; ++L) {
        const int N = 1 << L;
        std::vector<float2> tw = twiddles(L);
        std::vector<double> xr(NB * N), xi(NB * N);
        for (int n = 0; n < NB * N; ++n) {
            xr[n] = rand() / (double)RAND_MAX - 0.5;
            xi[n] = rand() / (double)RAND_MAX - 0.5;
        }
        double worst[8] = {0};
        for (int kind = 0; kind < 8; ++kind) {
            const bool inv = kind & 1;      // sign +
            const bool dit = kind & 2;      // bit-reversed in, natural out
            const bool split = kind & 4;
            const int ldi = ld_interleaved(N), lds = ld_split(N);
            std::vector<float2> ibuf((size_t)NB * ldi);
            std::vector<float> re((size_t)NB * lds), im((size_t)NB * lds);
            IBatch ib{ibuf.data(), ldi};
            SBatch sb{re.data(), im.data(), lds};
            for (int b = 0; b < NB; ++b)
                for (int n = 0; n < N; ++n) {
                    const int pos = dit ? (int)brev_bits(n, L) : n;
                    const float2 v = make_float2((float)xr[b * N + n], (float)xi[b * N + n]);
                    if (split) sb(b).st(pos, v); else ib(b).st(pos, v);
                }
#define RUN(D, I) \
    do { if (split) run<D, I>(sb, NB, L, tw.data()); else run<D, I>(ib, NB, L, tw.data()); } while (0)
            if (!dit && !inv) RUN(true, false);
            if (!dit && inv) RUN(true, true);
            if (dit && !inv) RUN(false, false);
            if (dit && inv) RUN(false, true);
#undef RUN
            double num = 0, den = 0;
            for (int b = 0; b < NB; ++b)
                for (int k = 0; k < N; ++k) {
                    double sr = 0, si = 0;
                    const double sg = inv ? 2.0 : -2.0;
                    for (int n = 0; n < N; ++n) {
                        const double a = sg * M_PI * (double)((long long)k * n % N) / N;
                        sr += xr[b * N + n] * cos(a) - xi[b * N + n] * sin(a);
                        si += xr[b * N + n] * sin(a) + xi[b * N + n] * cos(a);
                    }
                    const int pos = dit ? k : (int)brev_bits(k, L);
                    const float2 g = split ? sb(b).ld(pos) : ib(b).ld(pos);
                    num += (g.x - sr) * (g.x - sr) + (g.y - si) * (g.y - si);
                    den += sr * sr + si * si;
                }
            worst[kind] = sqrt(num / den);
            if (worst[kind] > worst_all) worst_all = worst[kind];
        }
        printf("N=%5d", N);
        for (int kind = 0; kind < 8; ++kind) printf(" %.1e", worst[kind]);
        printf("\n");
    }
    printf("worst %.3e\n", worst_all);
    return worst_all < 1e-5 ? 0 : 1;
}
