// Host build of the kernels' FP32 Faddeeva evaluation (faddeeva.cuh): reads
// "a x" pairs from stdin and prints H, Im w, dH/da and dH/dx for each.
#include <cstdio>
#include "faddeeva.cuh"

int main() {
    double a, x;
    while (std::scanf("%lf %lf", &a, &x) == 2) {
        const float xh = (float)x, xl = (float)(x - (double)xh);
        float H, K, H2, Ha, Hx;
        rg::faddeeva_hk((float)a, xh, xl, H, K);
        rg::faddeeva_derivs((float)a, (float)x, H2, Ha, Hx);
        std::printf("%.9e %.9e %.9e %.9e\n", H, K, Ha, Hx);
    }
    return 0;
}
