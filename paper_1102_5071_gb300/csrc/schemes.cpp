// Host-side CFET scheme data: coefficient tables, rule (R1) expansion,
// Gauss-Legendre rules and the quadrature coefficients g_{i,m}.
//
// Alvermann & Fehske, arXiv:1102.5071:
//   tables    Sec. 4.2 (Table 4thCFET), 4.3 (Table 6thCFET), 4.4 (Table
//             8thCoeff), 5.2 (Table 4thCFETOpt), 5.3 (Table 6thCFETOpt)
//   rule R1   Eq. (FSymm), Sec. 4.1: f_{s-i+1,n} = (-1)^{n+1} f_{i,n}
//   GL rule   Table tab:GaussLeg, Sec. 7
//   g_{i,m}   Sec. 7, after Eq. (OmGLeg):
//             g_{i,m} = w_m sum_n (2n-1) P_{n-1}(x_m) f_{i,n}
//   P_n       shifted Legendre recurrence, Sec. 3.1
#include <cmath>
#include <cstring>

#include "cfet_internal.h"

namespace cfet {
namespace {

// Shifted Legendre polynomial on [0,1] by the three-term recurrence.
double legendre01(int n, double x) {
  double p0 = 1.0;
  if (n == 0) return p0;
  double t = 2.0 * x - 1.0;
  double p1 = t;
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

void gl_rule(int M, double* x, double* w) {
  switch (M) {
    case 1:
      x[0] = 0.5; w[0] = 1.0;
      break;
    case 2: {
      const double d = std::sqrt(3.0) / 6.0;
      x[0] = 0.5 - d; x[1] = 0.5 + d;
      w[0] = w[1] = 0.5;
      break;
    }
    case 3: {
      const double d = std::sqrt(0.15);  // sqrt(3/20)
      x[0] = 0.5 - d; x[1] = 0.5; x[2] = 0.5 + d;
      w[0] = w[2] = 5.0 / 18.0; w[1] = 4.0 / 9.0;
      break;
    }
    default: {  // M == 4
      const double q = 2.0 * std::sqrt(1.2);  // 2 sqrt(6/5)
      const double a = std::sqrt((3.0 + q) / 28.0), b = std::sqrt((3.0 - q) / 28.0);
      x[0] = 0.5 - a; x[1] = 0.5 - b; x[2] = 0.5 + b; x[3] = 0.5 + a;
      const double r = std::sqrt(30.0);
      w[0] = w[3] = (18.0 - r) / 72.0;
      w[1] = w[2] = (18.0 + r) / 72.0;
      break;
    }
  }
}

// A printed half table: `rows` rows of `nA` entries (f_{i,1..nA}).
struct HalfTable {
  int order, s, nA, rows;
  double f[6][4];
};

bool half_table(int id, HalfTable* t) {
  std::memset(t, 0, sizeof(*t));
  switch (id) {
    case CFET_SCHEME_CF2_1:
      *t = {2, 1, 1, 1, {{1.0}}};
      return true;
    case CFET_SCHEME_CF4_2:
      *t = {4, 2, 2, 1, {{0.5, 1.0 / 3.0}}};
      return true;
    case CFET_SCHEME_CF4_3:
      *t = {4, 3, 2, 2, {{11.0 / 40.0, 20.0 / 87.0}, {9.0 / 20.0, 0.0}}};
      return true;
    case CFET_SCHEME_CF4_3OPT:
      *t = {4, 3, 3, 2, {{11.0 / 40.0, 20.0 / 87.0, 7.0 / 50.0}, {9.0 / 20.0, 0.0, -7.0 / 25.0}}};
      return true;
    case CFET_SCHEME_CF6_4: {
      // closed form of Table 6thCFET; the central exponentials vanish
      const double r6 = std::sqrt(6.0);
      const double a = 0.5 + std::cbrt(5400.0 - 600.0 * r6) / 60.0 +
                       std::cbrt((9.0 + r6) / 5.0) / (2.0 * std::pow(3.0, 2.0 / 3.0));
      const double c = 1.0 / (10.0 - 10.0 * a);
      *t = {6, 4, 3, 2, {{a, a - 2.0 * a * a / 3.0, c}, {0.5 - a, (1.0 - 4.0 * a + 2.0 * a * a) / 3.0, -c}}};
      return true;
    }
    case CFET_SCHEME_CF6_5:
    case CFET_SCHEME_CF6_5B:
    case CFET_SCHEME_CF6_5IMP:
    case CFET_SCHEME_CF6_5OPT: {
      // s = 5: rows 1, 2 printed; central row f31 = 1 - 2 f21 - 2 f11,
      // f32 = 0, f33 = -2 f23 - 2 f13, f34 = 0
      double r1[4] = {0, 0, 0, 0}, r2[4] = {0, 0, 0, 0};
      int nA = 3;
      if (id == CFET_SCHEME_CF6_5 || id == CFET_SCHEME_CF6_5IMP) {
        r1[0] = 0.16; r1[1] = 0.14587456942714338561; r1[2] = 0.11762370828143015682;
        r2[0] = 0.38752405202531186588; r2[1] = 0.15089113704380764664; r2[2] = -0.12805075909013044594;
        if (id == CFET_SCHEME_CF6_5IMP) { nA = 4; r1[3] = 0.074; r2[3] = -0.212530296697694739551; }
      } else if (id == CFET_SCHEME_CF6_5B) {
        r1[0] = 0.2; r1[1] = 0.1746879190177786220; r1[2] = 0.12406375705333586606;
        r2[0] = 0.34815492558797391479; r2[1] = 0.1068765450953683; r2[2] = -0.139021313323765096675;
      } else {
        nA = 4;
        r1[0] = 0.1714; r1[1] = 0.15409059414309687213; r1[2] = 0.11947178242929061641; r1[3] = 0.07195;
        r2[0] = 0.37496374319946236513; r2[1] = 0.13813675394387646682; r2[2] = -0.13090674649282935743;
        r2[3] = -0.21123356253315514306;
      }
      t->order = 6; t->s = 5; t->nA = nA; t->rows = 3;
      for (int n = 0; n < 4; ++n) { t->f[0][n] = r1[n]; t->f[1][n] = r2[n]; }
      t->f[2][0] = 1.0 - 2.0 * r2[0] - 2.0 * r1[0];
      t->f[2][1] = 0.0;
      t->f[2][2] = -2.0 * r2[2] - 2.0 * r1[2];
      t->f[2][3] = 0.0;
      return true;
    }
    case CFET_SCHEME_CF6_6: {
      const double a[3] = {0.16, 0.15101538937746543493, 0.13304616813239630479};
      const double b[3] = {-0.22738164742696330169, -0.087654259755115431662, 0.069919836812656575583};
      *t = {6, 6, 3, 3, {{a[0], a[1], a[2]}, {b[0], b[1], b[2]},
                          {0.5 - a[0] - b[0], 0.21035154512209824847, -a[2] - b[2]}}};
      return true;
    }
    case CFET_SCHEME_CF6_6OPT: {
      const double a[4] = {0.3952, 0.35629343479227292880, 0.27848030437681878641, 0.1579};
      const double b[4] = {-0.22432144875476807927, -0.19935407393749030416, -0.15625650102884866893, -0.09512};
      *t = {6, 6, 4, 3, {{a[0], a[1], a[2], a[3]}, {b[0], b[1], b[2], b[3]},
                          {0.5 - a[0] - b[0], 0.1145, -a[2] - b[2], -0.16475168057141371958}}};
      return true;
    }
    case CFET_SCHEME_CF8_11:
      *t = {8, 11, 4, 6, {
          {0.169715531043933180094151, 0.152866146944615909929839, 0.119167378745981369601216, 0.068619226448029559107538},
          {0.379420807516005431504230, 0.148839980923180990943008, -0.115880829186628075021088, -0.188555246668412628269760},
          {0.469459306644050573017994, -0.379844237839363505173921, 0.022898814729462898505141, 0.571855043580130805495594},
          {-0.448225927391070886302766, 0.362889857410989942809900, -0.022565582830528472333301, -0.544507517141613383517695},
          {-0.293924473106317605373923, -0.026255628265819381983204, 0.096761509131620390100068, 0.000018330145571671744069},
          {0.447109510586798614120629, 0.0, -0.200762581179816221704073, 0.0}}};
      return true;
    default:
      return false;
  }
}

}  // namespace

int default_scheme_for_order(int order) {
  switch (order) {
    case 2: return CFET_SCHEME_CF2_1;
    case 4: return CFET_SCHEME_CF4_2;
    case 6: return CFET_SCHEME_CF6_5OPT;
    case 8: return CFET_SCHEME_CF8_11;
    default: return 0;
  }
}

bool build_scheme(int id, SchemeData* out) {
  HalfTable t;
  if (!half_table(id, &t)) return false;
  std::memset(out, 0, sizeof(*out));
  out->id = id;
  out->order = t.order;
  out->s = t.s;
  out->M = t.nA;
  // rule (R1): mirror rows with sign (-1)^{n+1}, n 1-based
  for (int i = 0; i < t.rows; ++i) {
    for (int n = 0; n < t.nA; ++n) {
      out->f[i][n] = t.f[i][n];
      const int mirror = t.s - 1 - i;
      if (mirror != i) out->f[mirror][n] = ((n % 2) == 0 ? 1.0 : -1.0) * t.f[i][n];
    }
  }
  gl_rule(out->M, out->x, out->w);
  for (int i = 0; i < t.s; ++i) {
    for (int m = 0; m < out->M; ++m) {
      double acc = 0.0;
      for (int n = 1; n <= t.nA; ++n) acc += (2.0 * n - 1.0) * legendre01(n - 1, out->x[m]) * out->f[i][n - 1];
      out->g[i][m] = out->w[m] * acc;
    }
  }
  return true;
}

}  // namespace cfet
