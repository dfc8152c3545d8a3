// Host build of the kernels' integer exponential, logarithm, reciprocal, square root, sine/cosine
// and running product (fexp_scaled, flog, frcp, fsqrt, fsincos_pi, LogProd) for their accuracy
// tests: `math_host exp|log|rcp|sqrt in.bin out.bin` applies the function, with the device table's contents, to the
// doubles of in.bin (`sincos` writes sin x, cos x for each);
// `math_host lprod ...` writes ln of the product of each run of 64 inputs (logprod_mul, then
// logprod_value); `math_host logtab - out.bin` writes the logarithm's table words followed by
// ln_ratio_q115(2, 1) and the kLn2Q115 constant (high word, low word each).
#include <stdio.h>
#include <string.h>

#include <vector>

#include "fp64_math.cuh"

int main(int argc, char** argv)
{
    if (argc != 4) return 2;
    const char* fn = argv[1];
    std::vector<double> tab(gbnll::kTabDoubles);
    gbnll::fill_device_tables(tab.data());
    if (strcmp(fn, "logtab") == 0) {
        std::vector<uint64_t> w(3 * gbnll::kLogSteps + 4);
        memcpy(w.data(), tab.data() + gbnll::kLogOffset, sizeof(uint64_t) * 3 * gbnll::kLogSteps);
        const unsigned __int128 l2 = gbnll::ln_ratio_q115(2, 1);
        w[3 * gbnll::kLogSteps] = (uint64_t)(l2 >> 64);
        w[3 * gbnll::kLogSteps + 1] = (uint64_t)l2;
        w[3 * gbnll::kLogSteps + 2] = gbnll::kLn2Q115Hi;
        w[3 * gbnll::kLogSteps + 3] = gbnll::kLn2Q115Lo;
        FILE* o = fopen(argv[3], "wb");
        if (!o) return 4;
        const size_t n = fwrite(w.data(), sizeof(uint64_t), w.size(), o);
        fclose(o);
        return n == w.size() ? 0 : 5;
    }
    const bool is_exp = strcmp(fn, "exp") == 0, is_lprod = strcmp(fn, "lprod") == 0, is_log = strcmp(fn, "log") == 0;
    const bool is_sincos = strcmp(fn, "sincos") == 0, is_sqrt = strcmp(fn, "sqrt") == 0;
    if (!is_exp && !is_lprod && !is_log && !is_sincos && !is_sqrt && strcmp(fn, "rcp") != 0) return 2;
    FILE* f = fopen(argv[2], "rb");
    if (!f) return 3;
    std::vector<double> x;
    double v;
    while (fread(&v, sizeof v, 1, f) == 1) x.push_back(v);
    fclose(f);
    if (is_sincos) {
        std::vector<double> out(2 * x.size());
        for (size_t i = 0; i < x.size(); ++i)
            gbnll::fsincos_pi(x[i], tab.data() + gbnll::kTrigOffset, out[2 * i], out[2 * i + 1]);
        x.swap(out);
    } else if (is_lprod) {
        std::vector<double> out;
        for (size_t i = 0; i + 64 <= x.size(); i += 64) {
            gbnll::LogProd lp = gbnll::logprod_one();
            for (size_t k = 0; k < 64; ++k) gbnll::logprod_mul(lp, x[i + k]);
            out.push_back(gbnll::logprod_value(lp));
        }
        x.swap(out);
    } else {
        for (double& e : x)
            e = is_exp   ? gbnll::fexp_scaled(e, tab.data())
                : is_log ? gbnll::flog(e, tab.data())
                : is_sqrt ? gbnll::fsqrt(e)
                         : gbnll::frcp(e);
    }
    f = fopen(argv[3], "wb");
    if (!f) return 4;
    const size_t n = fwrite(x.data(), sizeof(double), x.size(), f);
    fclose(f);
    return n == x.size() ? 0 : 5;
}
