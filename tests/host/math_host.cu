// Host build of the kernels' integer exponential and reciprocal (fexp_scaled, frcp) for their
// accuracy tests: `math_host exp|rcp in.bin out.bin` applies the function, with the device
// table's contents, to the doubles of in.bin.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "fp64_math.cuh"

int main(int argc, char** argv)
{
    if (argc != 4) return 2;
    const bool is_exp = strcmp(argv[1], "exp") == 0;
    if (!is_exp && strcmp(argv[1], "rcp") != 0) return 2;
    FILE* f = fopen(argv[2], "rb");
    if (!f) return 3;
    std::vector<double> x;
    double v;
    while (fread(&v, sizeof v, 1, f) == 1) x.push_back(v);
    fclose(f);
    std::vector<double> tab(gbnll::kTabDoubles);
    gbnll::fill_device_tables(tab.data());
    for (double& e : x) e = is_exp ? gbnll::fexp_scaled(e, tab.data()) : gbnll::frcp(e);
    f = fopen(argv[3], "wb");
    if (!f) return 4;
    const size_t n = fwrite(x.data(), sizeof(double), x.size(), f);
    fclose(f);
    return n == x.size() ? 0 : 5;
}
