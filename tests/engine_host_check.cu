// engine_host_check.cu -- runs the FFT engine's stage code (fft_engine.cuh,
// host-callable) on the CPU against a direct DFT in long double, for every
// line shape the passes instantiate, in FP32, FP64 and float pairs.
//
// Built and run by tests/test_engine_host.py (host code only; no GPU).
// Prints one line per case: "<name> <max error / max |X|>".
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <complex>
#include <vector>

#include "fft_engine.cuh"

using namespace isofft;
typedef std::complex<long double> CL;

template <typename T>
static long double to_ld(T v)
{
    return (long double)v;
}
template <>
long double to_ld<df64>(df64 v)
{
    return (long double)v.hi + (long double)v.lo;
}
template <typename T>
static T from_d(double d)
{
    return (T)d;
}
template <>
df64 from_d<df64>(double d)
{
    return df64(d);
}

static const long double PI_L = 3.141592653589793238462643383279502884L;

static CL root(long n, long k)  // e^{-2 pi i k / n}
{
    const long double a = -2.0L * PI_L * (long double)(k % n) / (long double)n;
    return CL(cosl(a), sinl(a));
}

// twiddle table W_L^k, k < L, rounded from long double
template <typename T>
static std::vector<Cx<T>> table(int L)
{
    std::vector<Cx<T>> tw(L);
    for (int k = 0; k < L; ++k) {
        const CL w = root(L, k);
        tw[k] = {from_d<T>((double)w.real()), from_d<T>((double)w.imag())};
    }
    return tw;
}

// Host driver of a Radices<...> plan: every thread's stage, then the
// exchange the passes do through shared memory (write out_pos, read
// t + m NT), for all threads of the line.
template <typename T, int L, int E, int NS, bool HALF, int R, int... Rest>
static void drive(std::vector<Cx<T>> &pos, const Cx<T> *tw)
{
    constexpr int NT = L / E;
    using G = StageGeom<L, E, NS, R>;
    std::vector<Cx<T>> out(L);
    for (int t = 0; t < NT; ++t) {
        Cx<T> v[E];
        for (int m = 0; m < E; ++m) v[m] = pos[t + m * NT];
        stage<T, L, E, NS, R, HALF>(v, t, tw);
        for (int q = 0; q < G::B; ++q)
            for (int r = 0; r < R; ++r) out[G::out_pos(t, q, r)] = v[q + r * G::B];
    }
    pos = out;
    if constexpr (sizeof...(Rest) > 0) drive<T, L, E, NS * R, false, Rest...>(pos, tw);
}
template <typename T, int L, int E, bool HALF, int... Rs>
static void run_plan(std::vector<Cx<T>> &pos, const Cx<T> *tw, Radices<Rs...>)
{
    drive<T, L, E, 1, HALF, Rs...>(pos, tw);
}

// One shape: a random line (upper half zero when HALF), transformed by the
// plan, against the direct DFT.
template <typename T, int L, int E, typename Rad, bool HALF>
static void check_shape(const char *name, unsigned seed)
{
    srand(seed);
    std::vector<Cx<T>> x(L);
    std::vector<CL> xl(L);
    for (int i = 0; i < L; ++i) {
        double a = HALF && i >= L / 2 ? 0.0 : (double)rand() / RAND_MAX - 0.5;
        double b = HALF && i >= L / 2 ? 0.0 : (double)rand() / RAND_MAX - 0.5;
        x[i] = {from_d<T>(a), from_d<T>(b)};
        xl[i] = CL(to_ld(x[i].x), to_ld(x[i].y));
    }
    const std::vector<Cx<T>> tw = table<T>(L);
    run_plan<T, L, E, HALF>(x, tw.data(), Rad{});
    long double emax = 0, xmax = 0;
    for (int k = 0; k < L; ++k) {
        CL s = 0;
        for (int j = 0; j < L; ++j) s += xl[j] * root(L, (long)j * k);
        const CL got(to_ld(x[k].x), to_ld(x[k].y));
        emax = fmaxl(emax, std::abs(got - s));
        xmax = fmaxl(xmax, std::abs(s));
    }
    printf("%s %.3Le\n", name, emax / xmax);
}

template <typename T, typename SH, int L>
static void check(const char *tag, const char *kind, unsigned seed)
{
    char name[96];
    snprintf(name, sizeof name, "%s_%s_%d", kind, tag, L);
    check_shape<T, L, SH::E, typename SH::Rad, false>(name, seed);
    snprintf(name, sizeof name, "%s_%s_%d_half", kind, tag, L);
    check_shape<T, L, SH::E, typename SH::Rad, true>(name, seed + 1);
}

template <typename T>
static void check_all(const char *tag)
{
#define SH(S, L) check<T, S, L>(tag, #S, L);
    // column and z lines (Shape), every length the passes instantiate
    check<T, Shape<T, 32>, 32>(tag, "col", 1);
    check<T, Shape<T, 48>, 48>(tag, "col", 2);
    check<T, Shape<T, 64>, 64>(tag, "col", 3);
    check<T, Shape<T, 96>, 96>(tag, "col", 4);
    check<T, Shape<T, 128>, 128>(tag, "col", 5);
    check<T, Shape<T, 192>, 192>(tag, "col", 6);
    check<T, Shape<T, 256>, 256>(tag, "col", 7);
    check<T, Shape<T, 384>, 384>(tag, "col", 8);
    check<T, Shape<T, 512>, 512>(tag, "col", 9);
    check<T, Shape<T, 768>, 768>(tag, "col", 10);
    check<T, Shape<T, 1024>, 1024>(tag, "col", 11);
    check<T, Shape<T, 1536>, 1536>(tag, "col", 12);
    check<T, Shape<T, 2304>, 2304>(tag, "col", 13);
    // z-pass shapes
    check<T, ZShape<T, 384>, 384>(tag, "z", 27);
    check<T, ZShape<T, 512>, 512>(tag, "z", 14);
    check<T, ZShape<T, 768>, 768>(tag, "z", 15);
    check<T, ZShape<T, 2304>, 2304>(tag, "z", 16);
    check<T, ZShape<T, 128>, 128>(tag, "z", 28);
    check<T, ZShape<T, 192>, 192>(tag, "z", 29);
    check<T, ZShape<T, 256>, 256>(tag, "z", 30);
    check<T, ZShape<T, 1024>, 1024>(tag, "z", 31);
    // x rows (half-length complex transforms of the real rows)
    check<T, XShape<T, 16>, 16>(tag, "x", 17);
    check<T, XShape<T, 24>, 24>(tag, "x", 18);
    check<T, XShape<T, 256>, 256>(tag, "x", 19);
    check<T, XShapeF<T, 768>, 768>(tag, "xf", 20);
    check<T, XShapeF<T, 1152>, 1152>(tag, "xf", 21);
    check<T, XShape<T, 1152>, 1152>(tag, "x", 22);
    // the y passes' own shapes (FP32: 48 points a thread on 384- and
    // 2304-point lines, 32 on 512 and 1024, 24 on 192, 768 and 1536, 16 on
    // 256)
    check<T, YShape<T, 512>, 512>(tag, "y", 32);
    check<T, YShape<T, 1024>, 1024>(tag, "y", 33);
    check<T, YShape<T, 256>, 256>(tag, "y", 35);
    check<T, YShape<T, 192>, 192>(tag, "y", 36);
    check<T, XShapeF<T, 512>, 512>(tag, "xf", 34);
    check<T, YShape<T, 384>, 384>(tag, "y", 23);
    check<T, YShape<T, 768>, 768>(tag, "y", 24);
    check<T, YShape<T, 1536>, 1536>(tag, "y", 25);
    check<T, YShape<T, 2304>, 2304>(tag, "y", 26);
#undef SH
}

int main()
{
    check_all<float>("f32");
    check_all<double>("f64");
    check_all<df64>("df64");
    return 0;
}
