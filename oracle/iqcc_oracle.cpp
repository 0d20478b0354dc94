/*
 * TEST INFRASTRUCTURE.  Plain, slow, single-threaded CPU oracle for the iQCC
 * dressing path of arXiv 2603.08883.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the product path never does.
 * It shares no code with the CUDA library.
 *
 * Representation: a Pauli string is a std::string of letters 'I','X','Y','Z'
 * (qubit j at position j); the Hamiltonian is a hash map string -> real
 * coefficient (Eq. 2 / Eq. 9, real C_k).  Products are formed qubit by qubit
 * from the single-qubit letter table (XY = iZ, YZ = iX, ZX = iY, reversed
 * order gives -i, squares give I); there are no bit tricks here.
 *
 * Conventions (the library's, see the header of the CUDA library):
 *   dress(P, tau) maps H to e^{-i tau P/2} H e^{+i tau P/2}.  This is Eq. 5
 *   with the paper's amplitude tau_paper = -tau, so dress() evaluates Eq. 5
 *   literally at tau_paper = -tau.
 *   gradient(P) = dE/dtau at tau = 0 in that convention = -Im<Omega|H P|Omega>
 *   (Eq. 7 / Eq. 13 evaluate Im<Omega|H P|Omega> = dE/dtau_paper).
 *
 * Functions and the passages they follow:
 *   orc_load      Eq. 2 (sum of duplicate strings, exact zeros dropped)
 *   orc_dress     Eq. 5 / Eq. 6 (one generator)
 *   orc_energy    Eq. 3 / Eq. 10 / Eq. 12 at tau = 0 (QMF product state)
 *   orc_abc       Eq. 5 inserted into Eq. 12: E(tau) = A + B cos tau + C sin tau
 *   orc_gradient  Eq. 7 / Eq. 13
 *   orc_dis       App. A "Direct Interaction Space" (odd-Y, matching flip set),
 *                 Eq. 14-15 restriction when Omega is a z-eigenstate
 *   orc_prune     App. A procedure step 5 (compress small terms) and the
 *                 "Maximum Terms" limit of Tables 2-3
 *   orc_iterate   App. A procedure steps 1-5, one iteration
 *   orc_energy_gradients
 *                 derivatives of Eq. 12 (after Eq. 5 for one generator) with
 *                 respect to the Eq. 3 angles theta_j, phi_j and to tau
 */
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

namespace {

typedef std::complex<double> cplx;
typedef std::unordered_map<std::string, double> RealMap;
typedef std::unordered_map<std::string, cplx> CplxMap;

struct Oracle {
    int n;
    RealMap H;
};

/* ---------------- single-qubit algebra ---------------- */

int letter_index(char l) {
    switch (l) {
        case 'I': return 0;
        case 'X': return 1;
        case 'Y': return 2;
        default:  return 3; /* 'Z' */
    }
}
const char LETTERS[4] = {'I', 'X', 'Y', 'Z'};

/* a * b = i^power * letter */
struct LetterProduct { char letter; int power; };
const LetterProduct PRODUCT[4][4] = {
    /*        I          X          Y          Z     */
    /* I */ {{'I', 0}, {'X', 0}, {'Y', 0}, {'Z', 0}},
    /* X */ {{'X', 0}, {'I', 0}, {'Z', 1}, {'Y', 3}},
    /* Y */ {{'Y', 0}, {'Z', 3}, {'I', 0}, {'X', 1}},
    /* Z */ {{'Z', 0}, {'Y', 1}, {'X', 3}, {'I', 0}},
};

const cplx I_POW[4] = {cplx(1, 0), cplx(0, 1), cplx(-1, 0), cplx(0, -1)};

/* Product of two Pauli strings: a * b = i^power * out. */
int string_product(const std::string& a, const std::string& b, std::string& out) {
    out.assign(a.size(), 'I');
    int power = 0;
    for (size_t j = 0; j < a.size(); ++j) {
        const LetterProduct& p = PRODUCT[letter_index(a[j])][letter_index(b[j])];
        out[j] = p.letter;
        power += p.power;
    }
    return power & 3;
}

/* ---------------- key conversion and canonical order ---------------- */

std::string letters_from_bits(int n, const uint64_t* x, const uint64_t* z) {
    std::string s(n, 'I');
    for (int j = 0; j < n; ++j) {
        int xb = (int)((x[j / 64] >> (j % 64)) & 1u);
        int zb = (int)((z[j / 64] >> (j % 64)) & 1u);
        s[j] = LETTERS[xb ? (zb ? 2 : 1) : (zb ? 3 : 0)];
    }
    return s;
}

void bits_from_letters(const std::string& s, int W, uint64_t* x, uint64_t* z) {
    for (int w = 0; w < W; ++w) { x[w] = 0; z[w] = 0; }
    for (size_t j = 0; j < s.size(); ++j) {
        char l = s[j];
        if (l == 'X' || l == 'Y') x[j / 64] |= (uint64_t)1 << (j % 64);
        if (l == 'Z' || l == 'Y') z[j / 64] |= (uint64_t)1 << (j % 64);
    }
}

bool has_x(char l) { return l == 'X' || l == 'Y'; }
bool has_z(char l) { return l == 'Z' || l == 'Y'; }

/* Canonical order: the x bits as an unsigned integer (qubit n-1 most
   significant), then the z bits likewise. */
bool canonical_less(const std::string& a, const std::string& b) {
    for (size_t j = a.size(); j-- > 0;)
        if (has_x(a[j]) != has_x(b[j])) return !has_x(a[j]);
    for (size_t j = a.size(); j-- > 0;)
        if (has_z(a[j]) != has_z(b[j])) return !has_z(a[j]);
    return false;
}

/* ---------------- QMF product state (Eq. 3) ---------------- */

/* <psi_j| sigma |psi_j> for sigma in {I,X,Y,Z}, with the single-qubit state
   psi_j = (cos(theta/2), e^{i phi} sin(theta/2)), by explicit 2x2 products. */
struct Bloch { double e[4]; };

std::vector<Bloch> qmf_expectations(int n, const double* theta, const double* phi) {
    const cplx SIG[4][2][2] = {
        {{1, 0}, {0, 1}},
        {{0, 1}, {1, 0}},
        {{0, cplx(0, -1)}, {cplx(0, 1), 0}},
        {{1, 0}, {0, -1}},
    };
    std::vector<Bloch> out(n);
    for (int j = 0; j < n; ++j) {
        cplx psi[2] = {cplx(std::cos(theta[j] / 2), 0),
                       std::polar(1.0, phi[j]) * std::sin(theta[j] / 2)};
        for (int s = 0; s < 4; ++s) {
            cplx acc = 0;
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) acc += std::conj(psi[r]) * SIG[s][r][c] * psi[c];
            out[j].e[s] = acc.real();
        }
    }
    return out;
}

double expectation(const std::string& s, const std::vector<Bloch>& b) {
    double v = 1.0;
    for (size_t j = 0; j < s.size(); ++j) v *= b[j].e[letter_index(s[j])];
    return v;
}

bool is_z_eigenstate(int n, const double* theta) {
    for (int j = 0; j < n; ++j)
        if (!(theta[j] == 0.0 || theta[j] == M_PI)) return false;
    return true;
}

/* ---------------- compensated sum ---------------- */

struct Neumaier {
    double s = 0.0, c = 0.0;
    void add(double v) {
        double t = s + v;
        if (std::fabs(s) >= std::fabs(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    double value() const { return s + c; }
};

/* ---------------- Eq. 5 ---------------- */

/* [H, P] = H P - P H as a complex Pauli map.  A string that commutes with P
   contributes nothing and is not stored (its phases i^a and i^b agree). */
CplxMap commutator(const RealMap& H, const std::string& P) {
    CplxMap out;
    std::string hp, ph;
    for (const auto& kv : H) {
        int a = string_product(kv.first, P, hp);
        int b = string_product(P, kv.first, ph);
        /* hp and ph are the same string; the coefficients are i^a and i^b */
        if (a != b) out[hp] += kv.second * (I_POW[a] - I_POW[b]);
    }
    return out;
}

CplxMap left_multiply(const std::string& P, const CplxMap& A) {
    CplxMap out;
    std::string pa;
    for (const auto& kv : A) {
        int a = string_product(P, kv.first, pa);
        out[pa] += I_POW[a] * kv.second;
    }
    return out;
}

struct Cand { std::string key; double g; };

/* See orc_dis. */
std::vector<Cand> dis_candidates(Oracle* o, const double* theta, const double* phi) {
    int n = o->n;
    std::vector<Bloch> b = qmf_expectations(n, theta, phi);
    bool zeig = is_z_eigenstate(n, theta);

    /* group terms by flip set */
    std::unordered_map<std::string, std::vector<const std::pair<const std::string, double>*>> groups;
    for (const auto& kv : o->H) {
        std::string flip(n, '0');
        bool any = false;
        for (int j = 0; j < n; ++j)
            if (has_x(kv.first[j])) { flip[j] = '1'; any = true; }
        if (any) groups[flip].push_back(&kv);
    }
    std::vector<Cand> cands;
    cands.reserve(groups.size());
    std::string tp;
    for (const auto& gr : groups) {
        std::string P(n, 'I');
        bool first = true;
        for (int j = 0; j < n; ++j)
            if (gr.first[j] == '1') { P[j] = first ? 'Y' : 'X'; first = false; }
        Neumaier g;
        if (zeig) {
            for (const auto* kv : gr.second) {
                int a = string_product(kv->first, P, tp);
                g.add(kv->second * I_POW[a].imag() * expectation(tp, b));
            }
        } else {
            for (const auto& kv : o->H) {
                int a = string_product(kv.first, P, tp);
                g.add(kv.second * I_POW[a].imag() * expectation(tp, b));
            }
        }
        cands.push_back({P, -g.value()});
    }
    auto coarse = [](double g) {
        double a = std::fabs(g);
        uint64_t u;
        std::memcpy(&u, &a, 8);
        u &= ~(((uint64_t)1 << 20) - 1);
        std::memcpy(&a, &u, 8);
        return a;
    };
    std::sort(cands.begin(), cands.end(), [&](const Cand& p, const Cand& q) {
        double a = coarse(p.g), c = coarse(q.g);
        if (a != c) return a > c;
        return canonical_less(p.key, q.key);
    });
    return cands;
}

}  // namespace

extern "C" {

void* orc_new(int n) {
    if (n <= 0) return nullptr;
    Oracle* o = new Oracle();
    o->n = n;
    return o;
}

void orc_free(void* h) { delete (Oracle*)h; }

int64_t orc_size(void* h) { return (int64_t)((Oracle*)h)->H.size(); }

/* Eq. 2: H = sum_k C_k P_k; repeated strings are summed, exact zeros dropped. */
int orc_load(void* h, int64_t m, const uint64_t* x, const uint64_t* z, const double* c) {
    Oracle* o = (Oracle*)h;
    int W = (o->n + 63) / 64;
    for (int64_t k = 0; k < m; ++k)
        o->H[letters_from_bits(o->n, x + k * W, z + k * W)] += c[k];
    for (auto it = o->H.begin(); it != o->H.end();)
        it = (it->second == 0.0) ? o->H.erase(it) : std::next(it);
    return 0;
}

/* Terms in canonical order.  Returns the count; copies min(count, cap) rows. */
int64_t orc_export(void* h, int64_t cap, uint64_t* x, uint64_t* z, double* c) {
    Oracle* o = (Oracle*)h;
    int W = (o->n + 63) / 64;
    std::vector<std::pair<std::string, double>> rows(o->H.begin(), o->H.end());
    std::sort(rows.begin(), rows.end(),
              [](const std::pair<std::string, double>& a, const std::pair<std::string, double>& b) {
                  return canonical_less(a.first, b.first);
              });
    for (int64_t k = 0; k < (int64_t)rows.size() && k < cap; ++k) {
        bits_from_letters(rows[k].first, W, x + k * W, z + k * W);
        c[k] = rows[k].second;
    }
    return (int64_t)rows.size();
}

/* One generator P with library amplitude tau (Eq. 5 at tau_paper = -tau):
     H_d = H - (i/2) sin(tau_p) [H,P] + 1/2 (1 - cos(tau_p)) P [H,P].
   Returns 0, or -1 when an imaginary part survives (it must not for a real H
   and a Hermitian P; checked to 1e-9 of the largest contribution). */
int orc_dress(void* h, const uint64_t* gx, const uint64_t* gz, double tau) {
    Oracle* o = (Oracle*)h;
    std::string P = letters_from_bits(o->n, gx, gz);
    double tau_p = -tau;
    CplxMap comm = commutator(o->H, P);
    CplxMap pcomm = left_multiply(P, comm);
    CplxMap out;
    for (const auto& kv : o->H) out[kv.first] += kv.second;
    cplx a = cplx(0, -0.5) * std::sin(tau_p);
    double b = 0.5 * (1.0 - std::cos(tau_p));
    for (const auto& kv : comm) out[kv.first] += a * kv.second;
    for (const auto& kv : pcomm) out[kv.first] += b * kv.second;
    double scale = 0.0, worst = 0.0;
    for (const auto& kv : out) {
        scale = std::max(scale, std::abs(kv.second));
        worst = std::max(worst, std::fabs(kv.second.imag()));
    }
    if (worst > 1e-9 * std::max(scale, 1e-300) && worst > 1e-300) return -1;
    o->H.clear();
    for (const auto& kv : out) o->H[kv.first] = kv.second.real();
    return 0;
}

/* Eq. 12 at tau = 0: E = sum_k C_k <Omega|P_k|Omega>, compensated sum. */
double orc_energy(void* h, const double* theta, const double* phi) {
    Oracle* o = (Oracle*)h;
    std::vector<Bloch> b = qmf_expectations(o->n, theta, phi);
    Neumaier s;
    for (const auto& kv : o->H) s.add(kv.second * expectation(kv.first, b));
    return s.value();
}

/* E(tau) = <Omega| e^{-i tau P/2} H e^{i tau P/2} |Omega> = A + B cos tau + C sin tau.
   From Eq. 5 (library sign): commuting strings give A; an anticommuting T gives
   cos(tau) <T> (into B) and sin(tau) <i T P> (into C). */
void orc_abc(void* h, const uint64_t* gx, const uint64_t* gz, const double* theta,
             const double* phi, double* abc) {
    Oracle* o = (Oracle*)h;
    std::string P = letters_from_bits(o->n, gx, gz);
    std::vector<Bloch> b = qmf_expectations(o->n, theta, phi);
    Neumaier A, B, C;
    std::string tp, pt;
    for (const auto& kv : o->H) {
        int a = string_product(kv.first, P, tp);
        int c = string_product(P, kv.first, pt);
        if (a == c) {                         /* T P = P T */
            A.add(kv.second * expectation(kv.first, b));
        } else {                              /* T P = -P T */
            B.add(kv.second * expectation(kv.first, b));
            cplx itp = cplx(0, 1) * I_POW[a]; /* i T P = itp * tp, itp = +-1 */
            C.add(kv.second * itp.real() * expectation(tp, b));
        }
    }
    abc[0] = A.value();
    abc[1] = B.value();
    abc[2] = C.value();
}

/* Eq. 7: g_paper = Im <Omega| H P |Omega>; returns the library-sign gradient
   dE/dtau = -g_paper. */
double orc_gradient(void* h, const uint64_t* gx, const uint64_t* gz, const double* theta,
                    const double* phi) {
    Oracle* o = (Oracle*)h;
    std::string P = letters_from_bits(o->n, gx, gz);
    std::vector<Bloch> b = qmf_expectations(o->n, theta, phi);
    Neumaier g;
    std::string tp;
    for (const auto& kv : o->H) {
        int a = string_product(kv.first, P, tp);
        g.add(kv.second * I_POW[a].imag() * expectation(tp, b));
    }
    return -g.value();
}

/* d<psi|sigma|psi>/d theta and d/d phi for sigma in {I,X,Y,Z}, as
   2 Re <d psi|sigma|psi> from explicit 2x2 products, with
   d psi/d theta = (-sin(theta/2)/2, e^{i phi} cos(theta/2)/2) and
   d psi/d phi = (0, i e^{i phi} sin(theta/2)). */
void qmf_derivatives(int n, const double* theta, const double* phi, std::vector<Bloch>& dth,
                     std::vector<Bloch>& dph) {
    const cplx SIG[4][2][2] = {
        {{1, 0}, {0, 1}},
        {{0, 1}, {1, 0}},
        {{0, cplx(0, -1)}, {cplx(0, 1), 0}},
        {{1, 0}, {0, -1}},
    };
    dth.assign(n, Bloch{});
    dph.assign(n, Bloch{});
    for (int j = 0; j < n; ++j) {
        const cplx e = std::polar(1.0, phi[j]);
        const cplx psi[2] = {cplx(std::cos(theta[j] / 2), 0), e * std::sin(theta[j] / 2)};
        const cplx d_t[2] = {cplx(-std::sin(theta[j] / 2) / 2, 0), e * std::cos(theta[j] / 2) / 2.0};
        const cplx d_p[2] = {cplx(0, 0), cplx(0, 1) * e * std::sin(theta[j] / 2)};
        for (int s = 0; s < 4; ++s) {
            cplx at = 0, ap = 0;
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) {
                    at += std::conj(d_t[r]) * SIG[s][r][c] * psi[c];
                    ap += std::conj(d_p[r]) * SIG[s][r][c] * psi[c];
                }
            dth[j].e[s] = 2.0 * at.real();
            dph[j].e[s] = 2.0 * ap.real();
        }
    }
}

/* E(tau) = <Omega| e^{-i tau P/2} H e^{+i tau P/2} |Omega> (Eq. 5 inserted into
   Eq. 12) and its derivatives with respect to the angles of Eq. 3 and to tau.
   Route: dress a copy of H by (P, tau) with orc_dress, then differentiate each
   string of the copy qubit by qubit (product rule: the derivative of qubit k's
   factor times the product of the other qubits' factors, by an explicit loop).
   dE/dtau = -B sin tau + C cos tau with A, B, C from orc_abc on H.  gx = gz =
   NULL: no generator (the energy of H and its angle gradient; d_tau = 0).
   Returns E(tau); d_theta, d_phi: n values each. */
double orc_energy_gradients(void* h, const uint64_t* gx, const uint64_t* gz, double tau, const double* theta,
                            const double* phi, double* d_theta, double* d_phi, double* d_tau) {
    Oracle* o = (Oracle*)h;
    Oracle work = *o;
    *d_tau = 0.0;
    if (gx && gz) {
        if (orc_dress(&work, gx, gz, tau) != 0) return std::nan("");
        double abc[3];
        orc_abc(h, gx, gz, theta, phi, abc);
        *d_tau = -abc[1] * std::sin(tau) + abc[2] * std::cos(tau);
    }
    const int n = o->n;
    std::vector<Bloch> b = qmf_expectations(n, theta, phi);
    std::vector<Bloch> dth, dph;
    qmf_derivatives(n, theta, phi, dth, dph);
    std::vector<Neumaier> gt(n), gp(n);
    Neumaier e;
    for (const auto& kv : work.H) {
        const std::string& s = kv.first;
        e.add(kv.second * expectation(s, b));
        for (int k = 0; k < n; ++k) {
            const int lk = letter_index(s[k]);
            if (lk == 0) continue;
            double others = 1.0;
            for (int j = 0; j < n; ++j)
                if (j != k) others *= b[j].e[letter_index(s[j])];
            gt[k].add(kv.second * dth[k].e[lk] * others);
            gp[k].add(kv.second * dph[k].e[lk] * others);
        }
    }
    for (int k = 0; k < n; ++k) {
        d_theta[k] = gt[k].value();
        d_phi[k] = gp[k].value();
    }
    return e.value();
}

/* DIS candidates: one representative per distinct non-empty flip set
   F = {j : letter in {X,Y}} of a term of H, with Y at the lowest qubit of F
   and X on the rest of F (odd Y parity, matching flip set; App. A).  Each
   gradient is Eq. 7 (library sign).  When every theta_j is 0 or pi the state
   is a z-eigenstate and only terms with the candidate's own flip set
   contribute (Eq. 14-15); otherwise every term is summed.
   Ordering: |g| with its 20 lowest mantissa bits cleared (a tie tolerance of
   about 2^-32 relative), descending, then the candidate's key ascending in
   canonical order.  Returns the count; copies min(count, cap) candidates. */
int64_t orc_dis(void* h, const double* theta, const double* phi, int64_t cap,
                uint64_t* ox, uint64_t* oz, double* grad) {
    Oracle* o = (Oracle*)h;
    int W = (o->n + 63) / 64;
    std::vector<Cand> cands = dis_candidates(o, theta, phi);
    for (int64_t k = 0; k < (int64_t)cands.size() && k < cap; ++k) {
        bits_from_letters(cands[k].key, W, ox + k * W, oz + k * W);
        grad[k] = cands[k].g;
    }
    return (int64_t)cands.size();
}

/* Compression: drop |c| < eps; then, if more than max_terms remain (and
   max_terms > 0), keep the max_terms largest |c|, ties broken towards the
   smaller key in canonical order.  Returns the number of removed terms. */
int64_t orc_prune(void* h, double eps, int64_t max_terms) {
    Oracle* o = (Oracle*)h;
    int64_t before = (int64_t)o->H.size();
    for (auto it = o->H.begin(); it != o->H.end();)
        it = (std::fabs(it->second) < eps) ? o->H.erase(it) : std::next(it);
    if (max_terms > 0 && (int64_t)o->H.size() > max_terms) {
        std::vector<std::pair<std::string, double>> rows(o->H.begin(), o->H.end());
        std::sort(rows.begin(), rows.end(),
                  [](const std::pair<std::string, double>& a, const std::pair<std::string, double>& b) {
                      if (std::fabs(a.second) != std::fabs(b.second))
                          return std::fabs(a.second) > std::fabs(b.second);
                      return canonical_less(a.first, b.first);
                  });
        o->H.clear();
        for (int64_t k = 0; k < max_terms; ++k) o->H[rows[k].first] = rows[k].second;
    }
    return before - (int64_t)o->H.size();
}

/* One iQCC iteration (App. A procedure):
     1. DIS gradients of all candidates (orc_dis order);
     2. the top n_gen candidates with |g| > 1e-12 (or the n_forced given ones);
     3. for each in turn: A, B, C on the current H and tau = atan2(-C, -B)
        (the minimiser of A + B cos tau + C sin tau; 0 when B = C = 0), or the
        given tau when tau_forced is not null; dress; when max_terms > 0 and
        the dressed H holds more than max_terms terms, keep the max_terms
        largest at once (the term limit holds after every dress);
     4. compress with (eps, max_terms);
     5. energy.
   Outputs: gens_x/gens_z [n_gen][W], g[n_gen], tau[n_gen], abc[n_gen][3];
   returns the number of generators applied, or -1 on error. */
int orc_iterate(void* h, const double* theta, const double* phi, int n_gen, int n_forced,
                const uint64_t* forced_x, const uint64_t* forced_z, const double* tau_forced,
                double eps, int64_t max_terms, uint64_t* gens_x, uint64_t* gens_z, double* g,
                double* tau, double* abc, int64_t* removed, double* energy) {
    Oracle* o = (Oracle*)h;
    int W = (o->n + 63) / 64;
    int used = 0;
    *removed = 0;
    if (n_forced > 0) {
        used = n_forced;
        for (int k = 0; k < used; ++k) {
            std::memcpy(gens_x + k * W, forced_x + k * W, 8 * W);
            std::memcpy(gens_z + k * W, forced_z + k * W, 8 * W);
            g[k] = orc_gradient(h, forced_x + k * W, forced_z + k * W, theta, phi);
        }
    } else {
        std::vector<Cand> cands = dis_candidates(o, theta, phi);
        for (size_t k = 0; k < cands.size() && used < n_gen; ++k) {
            if (!(std::fabs(cands[k].g) > 1e-12)) continue;
            bits_from_letters(cands[k].key, W, gens_x + used * W, gens_z + used * W);
            g[used] = cands[k].g;
            ++used;
        }
    }
    for (int k = 0; k < used; ++k) {
        orc_abc(h, gens_x + k * W, gens_z + k * W, theta, phi, abc + 3 * k);
        double B = abc[3 * k + 1], C = abc[3 * k + 2];
        if (tau_forced) tau[k] = tau_forced[k];
        else tau[k] = (B == 0.0 && C == 0.0) ? 0.0 : std::atan2(-C, -B);
        if (orc_dress(h, gens_x + k * W, gens_z + k * W, tau[k])) return -1;
        if (max_terms > 0 && (int64_t)o->H.size() > max_terms) *removed += orc_prune(h, 0.0, max_terms);
    }
    *removed += orc_prune(h, eps, max_terms);
    *energy = orc_energy(h, theta, phi);
    return used;
}

}  // extern "C"
