// Host check of the grouped spread lists built at plan creation: for random
// sample geometries (kernel widths 6 and 8, bin strides 8-64, one or two
// frames, grid sizes 64 and 96) the lists are gathered as the spread kernel
// gathers them (each group's entries in list order, each cell's products
// fused in that order) and every value of every cell is compared bit for
// bit with a direct scatter of the samples in ascending m.  Also checks the
// blob's word layout, the padding and range of every offset, that every
// cell is written exactly once, and the admission estimate's bound on the
// list size.  Built with -I <kernel sources>; prints OK and exits 0 on
// success.
#include "plan.cu"
#include <cstdio>
#include <random>
using namespace prop;
int main() {
  int fails = 0;
  for (int W : {6, 8})
    for (int cs : {8, 16, 32, 64})
      for (int T : {1, 2})
        for (int n : {96, 64}) {
          Plan p;
          p.n = n;
          p.W = W;
          p.cs = cs;
          p.T = T;
          p.L = 6;
          p.R = 40;
          p.N = n / 2;
          const int B = 7;
          p.M = B * p.L * p.R;
          p.blade_frame.resize(B);
          for (int b = 0; b < B; ++b) p.blade_frame[b] = b * T / B;
          std::mt19937 rng(W * 100 + cs + T + n);
          std::vector<int> first_tap(2 * p.M);
          std::vector<double> wd((size_t)p.M * 2 * W);
          for (int m = 0; m < p.M; ++m) {
            std::normal_distribution<double> nd(n / 2.0, n / 7.0);  // clustered, wrapping at the edges
            first_tap[2 * m] = ((int)nd(rng) % p.n + p.n) % p.n;
            first_tap[2 * m + 1] = ((int)nd(rng) % p.n + p.n) % p.n;
            for (int q = 0; q < 2 * W; ++q) wd[(size_t)m * 2 * W + q] = std::uniform_real_distribution<double>(0.1, 1.0)(rng);
          }
          std::vector<int4> sitems;
          std::vector<int2> blob;
          if (!build_group_lists(p, first_tap, wd, sitems, blob)) {
            printf("W%d cs%d T%d n%d: builder refused\n", W, cs, T, n);
            ++fails;
            continue;
          }
          std::vector<float> contrib((size_t)(p.M + 1) * cs * 2, 0.f);  // row M stays zero
          for (size_t i = 0; i < (size_t)p.M * cs * 2; ++i) contrib[i] = std::uniform_real_distribution<float>(-1, 1)(rng);
          const size_t ncell = (size_t)T * p.n * p.n;
          std::vector<float> ref(ncell * cs * 2, 0.f), got(ncell * cs * 2, -7.f);
          std::vector<int> writes(ncell, 0);
          const size_t LR = (size_t)p.L * p.R;
          for (int m = 0; m < p.M; ++m) {
            const size_t fr = p.blade_frame[m / LR];
            for (int a = 0; a < W; ++a)
              for (int b = 0; b < W; ++b) {
                const size_t cell = (fr * p.n + (first_tap[2 * m + 1] + a) % p.n) * p.n + (first_tap[2 * m] + b) % p.n;
                const float w = (float)(wd[(size_t)m * 2 * W + W + a] * wd[(size_t)m * 2 * W + b]);
                for (int f = 0; f < 2 * cs; ++f)
                  ref[cell * 2 * cs + f] = fmaf(w, contrib[(size_t)m * 2 * cs + f], ref[cell * 2 * cs + f]);
              }
          }
          for (const int4& it : sitems) {
            const int ng = it.y, nent = it.z, ngp = (ng + 1) & ~1;
            if (it.w > kSpreadStageInt2 || nent % 4 || (long)ngp + nent / 2 + 2L * nent != it.w ||
                (size_t)it.x + it.w > blob.size()) {
              printf("bad item layout\n");
              ++fails;
              continue;
            }
            const int2* base = &blob[it.x];
            const int* offs = reinterpret_cast<const int*>(base + ngp);
            const float* wts = reinterpret_cast<const float*>(base + ngp + nent / 2);
            for (int g = 0; g < ng; ++g) {
              const int cell0 = base[g].x, end = base[g].y, beg = g ? base[g - 1].y : 0;
              if ((end - beg) % 4 || end > nent || beg > end) {
                printf("list not padded or outside its item\n");
                ++fails;
                continue;
              }
              static float acc[4][128];
              for (int c = 0; c < 4; ++c)
                for (int f = 0; f < 2 * cs; ++f) acc[c][f] = 0.f;
              for (int e = beg; e < end; ++e) {
                if (offs[e] % cs || offs[e] / cs > p.M) {
                  printf("offset out of range\n");
                  ++fails;
                  break;
                }
                for (int c = 0; c < 4; ++c)
                  for (int f = 0; f < 2 * cs; ++f)
                    acc[c][f] = fmaf(wts[(size_t)4 * e + c], contrib[(size_t)offs[e] * 2 + f], acc[c][f]);
              }
              for (int c = 0; c < 4; ++c) {
                const size_t cell = (size_t)cell0 + (size_t)(c >> 1) * p.n + (c & 1);
                if (cell >= ncell) {
                  printf("cell out of range\n");
                  ++fails;
                  continue;
                }
                ++writes[cell];
                for (int f = 0; f < 2 * cs; ++f) got[cell * 2 * cs + f] = acc[c][f];
              }
            }
          }
          size_t bad = 0, twice = 0;
          for (size_t i = 0; i < ref.size(); ++i) bad += got[i] != ref[i];
          for (size_t c = 0; c < ncell; ++c) twice += writes[c] != 1;
          // the admission estimate's bound on the grouped lists (plan_estimate_bytes)
          const size_t bound = 8 * (ncell / 4) + 8 + (4 + 16) * 2 * 16 * (size_t)p.M + 16 * (ncell / 4);
          if (blob.size() * sizeof(int2) > bound) {
            printf("lists above the estimate's bound\n");
            ++fails;
          }
          printf("W%d cs%d T%d n%d: %zu items, %zu words, cells written other than once %zu, mismatching values %zu\n", W,
                 cs, T, n, sitems.size(), blob.size(), twice, bad);
          fails += bad != 0 || twice != 0;
        }
  printf(fails ? "FAIL\n" : "OK\n");
  return fails != 0;
}
