// qasm.cpp -- OpenQASM 2.0 text to gate records (qsim_parse_qasm).
//
// The paper's simulator takes circuits as OpenQASM files (Section "Simulator
// Framework": a QASM frontend feeding the gate table, Table "Gates defined in
// IBM OpenQASM").  This is a host-side reader for the OpenQASM 2.0 subset those
// files use: qreg / creg declarations, the qelib1 gate set (applied to single
// qubits or broadcast over whole registers), parameter expressions (pi,
// + - * / ^, unary minus, sin cos tan exp ln sqrt), user `gate` definitions
// (expanded like macros), measure / reset / barrier.  ccx, cswap, rccx and
// rc3x are decomposed into 1- and 2-qubit gates, c3x, c4x and c3sqrtx into
// controlled-X^t C2 records; sx / sxdg become C1 records.  Global
// phases follow the library's gate definitions (RZ(t) = exp(-i t Z/2),
// U3 as the standard three-angle matrix), as Qiskit's gates do.
#include <cctype>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/qsim.h"

namespace {

struct Tok {
    enum Kind { ID, NUM, STR, SYM, END } kind;
    std::string s;
    double v = 0;
    int line = 0;
};

struct ParseError : std::runtime_error {
    using std::runtime_error::runtime_error;
};

std::vector<Tok> lex(const char *p, size_t len) {
    std::vector<Tok> out;
    const char *e = p + len;
    int line = 1;
    while (p < e) {
        const char c = *p;
        if (c == '\n') {
            line++;
            p++;
        } else if (std::isspace((unsigned char)c)) {
            p++;
        } else if (c == '/' && p + 1 < e && p[1] == '/') {
            while (p < e && *p != '\n') p++;
        } else if (std::isalpha((unsigned char)c) || c == '_') {
            const char *b = p;
            while (p < e && (std::isalnum((unsigned char)*p) || *p == '_')) p++;
            out.push_back({Tok::ID, std::string(b, p), 0, line});
        } else if (std::isdigit((unsigned char)c) || (c == '.' && p + 1 < e && std::isdigit((unsigned char)p[1]))) {
            const char *b = p;
            while (p < e && (std::isdigit((unsigned char)*p) || *p == '.')) p++;
            if (p < e && (*p == 'e' || *p == 'E')) {
                p++;
                if (p < e && (*p == '+' || *p == '-')) p++;
                while (p < e && std::isdigit((unsigned char)*p)) p++;
            }
            const std::string s(b, p);
            out.push_back({Tok::NUM, s, std::strtod(s.c_str(), nullptr), line});
        } else if (c == '"') {
            const char *b = ++p;
            while (p < e && *p != '"' && *p != '\n') p++;
            if (p >= e || *p != '"') throw ParseError("line " + std::to_string(line) + ": unterminated string");
            out.push_back({Tok::STR, std::string(b, p), 0, line});
            p++;
        } else if (c == '-' && p + 1 < e && p[1] == '>') {
            out.push_back({Tok::SYM, "->", 0, line});
            p += 2;
        } else if (c == '=' && p + 1 < e && p[1] == '=') {
            out.push_back({Tok::SYM, "==", 0, line});
            p += 2;
        } else if (std::strchr("()[]{},;+-*/^", c)) {
            out.push_back({Tok::SYM, std::string(1, c), 0, line});
            p++;
        } else {
            throw ParseError("line " + std::to_string(line) + ": unexpected character '" + std::string(1, c) + "'");
        }
    }
    out.push_back({Tok::END, "", 0, line});
    return out;
}

// A parsed expression, evaluated against the parameters of a gate body.
struct Expr {
    enum Op { NUM, VAR, NEG, ADD, SUB, MUL, DIV, POW, FN } op = NUM;
    double v = 0;
    std::string name;  // VAR: parameter name; FN: function name
    std::shared_ptr<Expr> a, b;

    double eval(const std::map<std::string, double> &env) const {
        switch (op) {
            case NUM: return v;
            case VAR: {
                auto it = env.find(name);
                if (it == env.end()) throw ParseError("unknown parameter '" + name + "'");
                return it->second;
            }
            case NEG: return -a->eval(env);
            case ADD: return a->eval(env) + b->eval(env);
            case SUB: return a->eval(env) - b->eval(env);
            case MUL: return a->eval(env) * b->eval(env);
            case DIV: return a->eval(env) / b->eval(env);
            case POW: return std::pow(a->eval(env), b->eval(env));
            case FN: {
                const double x = a->eval(env);
                if (name == "sin") return std::sin(x);
                if (name == "cos") return std::cos(x);
                if (name == "tan") return std::tan(x);
                if (name == "exp") return std::exp(x);
                if (name == "ln") return std::log(x);
                if (name == "sqrt") return std::sqrt(x);
                throw ParseError("unknown function '" + name + "'");
            }
        }
        return 0;
    }
};
using ExprP = std::shared_ptr<Expr>;

// One operand of a gate application: a whole register (index < 0) or one qubit;
// inside a gate body, a formal argument.
struct Arg {
    std::string reg;
    long index = -1;
};

struct Stmt {
    std::string name;
    std::vector<ExprP> params;
    std::vector<Arg> args;
    int line = 0;
};

struct GateDef {
    std::vector<std::string> params, qargs;
    std::vector<Stmt> body;
};

class Parser {
  public:
    Parser(const char *text, size_t len) : t_(lex(text, len)) {}

    void run() {
        while (peek().kind != Tok::END) statement();
    }

    std::vector<qsim_gate> gates;
    std::vector<double> mats;
    int n_qubits = 0;

  private:
    std::vector<Tok> t_;
    size_t i_ = 0;
    std::map<std::string, std::pair<int, int>> qregs_;  // name -> (offset, size)
    std::map<std::string, int> cregs_;
    std::map<std::string, GateDef> defs_;
    int depth_ = 0;

    const Tok &peek() const { return t_[i_]; }
    [[noreturn]] void error(const std::string &m, int line = -1) const {
        throw ParseError("line " + std::to_string(line < 0 ? peek().line : line) + ": " + m);
    }
    bool is(const char *sym) const { return peek().kind == Tok::SYM && peek().s == sym; }
    void expect(const char *sym) {
        if (!is(sym)) error(std::string("expected '") + sym + "'");
        i_++;
    }
    std::string ident() {
        if (peek().kind != Tok::ID) error("expected an identifier");
        return t_[i_++].s;
    }
    long integer() {
        if (peek().kind != Tok::NUM) error("expected an integer");
        const double v = t_[i_++].v;
        if (v < 0 || v != std::floor(v)) error("expected an integer");
        return (long)v;
    }

    // expr := term (('+'|'-') term)*; term := unary (('*'|'/') unary)*;
    // unary := '-' unary | power; power := primary ('^' unary)?
    ExprP expr() {
        ExprP l = term();
        while (is("+") || is("-")) {
            auto n = std::make_shared<Expr>();
            n->op = t_[i_++].s == "+" ? Expr::ADD : Expr::SUB;
            n->a = l;
            n->b = term();
            l = n;
        }
        return l;
    }
    ExprP term() {
        ExprP l = unary();
        while (is("*") || is("/")) {
            auto n = std::make_shared<Expr>();
            n->op = t_[i_++].s == "*" ? Expr::MUL : Expr::DIV;
            n->a = l;
            n->b = unary();
            l = n;
        }
        return l;
    }
    ExprP unary() {
        if (is("-")) {
            i_++;
            auto n = std::make_shared<Expr>();
            n->op = Expr::NEG;
            n->a = unary();
            return n;
        }
        if (is("+")) {
            i_++;
            return unary();
        }
        ExprP p = primary();
        if (is("^")) {
            i_++;
            auto n = std::make_shared<Expr>();
            n->op = Expr::POW;
            n->a = p;
            n->b = unary();
            return n;
        }
        return p;
    }
    ExprP primary() {
        auto n = std::make_shared<Expr>();
        if (peek().kind == Tok::NUM) {
            n->v = t_[i_++].v;
            return n;
        }
        if (is("(")) {
            i_++;
            ExprP e = expr();
            expect(")");
            return e;
        }
        if (peek().kind == Tok::ID) {
            const std::string id = t_[i_++].s;
            if (id == "pi") {
                n->v = M_PI;
                return n;
            }
            if (is("(")) {
                i_++;
                n->op = Expr::FN;
                n->name = id;
                n->a = expr();
                expect(")");
                return n;
            }
            n->op = Expr::VAR;
            n->name = id;
            return n;
        }
        error("expected an expression");
    }

    Arg arg() {
        Arg a;
        a.reg = ident();
        if (is("[")) {
            i_++;
            a.index = integer();
            expect("]");
        }
        return a;
    }
    std::vector<Arg> arglist() {
        std::vector<Arg> v{arg()};
        while (is(",")) {
            i_++;
            v.push_back(arg());
        }
        return v;
    }

    void statement() {
        const int line = peek().line;
        if (peek().kind != Tok::ID) error("expected a statement");
        const std::string kw = peek().s;
        if (kw == "OPENQASM") {
            i_++;
            if (peek().kind != Tok::NUM || peek().v >= 3.0) error("only OpenQASM 2.x is read");
            i_++;
            expect(";");
        } else if (kw == "include") {
            i_++;
            if (peek().kind != Tok::STR) error("expected a file name");
            i_++;  // qelib1.inc is built in; other includes are not read
            expect(";");
        } else if (kw == "qreg" || kw == "creg") {
            i_++;
            const std::string name = ident();
            expect("[");
            const long size = integer();
            expect("]");
            expect(";");
            if (size <= 0) error("register size must be positive", line);
            if (qregs_.count(name) || cregs_.count(name)) error("register '" + name + "' declared twice", line);
            if (kw == "qreg") {
                qregs_[name] = {n_qubits, (int)size};
                n_qubits += (int)size;
                if (n_qubits > 64) error("more than 64 qubits", line);
            } else {
                cregs_[name] = (int)size;
            }
        } else if (kw == "gate") {
            i_++;
            const std::string name = ident();
            GateDef d;
            if (is("(")) {
                i_++;
                if (!is(")")) {
                    d.params.push_back(ident());
                    while (is(",")) {
                        i_++;
                        d.params.push_back(ident());
                    }
                }
                expect(")");
            }
            d.qargs.push_back(ident());
            while (is(",")) {
                i_++;
                d.qargs.push_back(ident());
            }
            expect("{");
            while (!is("}")) {
                if (peek().kind == Tok::END) error("unterminated gate body", line);
                Stmt s;
                s.line = peek().line;
                s.name = ident();
                if (s.name == "barrier") {  // no effect inside a gate body
                    arglist();
                    expect(";");
                    continue;
                }
                if (is("(")) {
                    i_++;
                    if (!is(")")) {
                        s.params.push_back(expr());
                        while (is(",")) {
                            i_++;
                            s.params.push_back(expr());
                        }
                    }
                    expect(")");
                }
                s.args = arglist();
                expect(";");
                d.body.push_back(s);
            }
            expect("}");
            defs_[name] = d;
        } else if (kw == "opaque" || kw == "if") {
            error("'" + kw + "' is not supported");
        } else if (kw == "measure") {
            i_++;
            const Arg q = arg();
            expect("->");
            const Arg c = arg();
            expect(";");
            if (!cregs_.count(c.reg)) error("unknown classical register '" + c.reg + "'", line);
            for (int qb : qubits(q, line)) push(QSIM_OP_MEASURE, qb, 0, 0, 0, 0);
        } else if (kw == "reset") {
            i_++;
            const Arg q = arg();
            expect(";");
            for (int qb : qubits(q, line)) push(QSIM_OP_RESET, qb, 0, 0, 0, 0);
        } else if (kw == "barrier") {
            i_++;
            for (const Arg &a : arglist()) qubits(a, line);  // validated; a barrier stops all reordering
            expect(";");
            push(QSIM_OP_BARRIER, 0, 0, 0, 0, 0);
        } else {
            Stmt s;
            s.line = line;
            s.name = ident();
            if (is("(")) {
                i_++;
                if (!is(")")) {
                    s.params.push_back(expr());
                    while (is(",")) {
                        i_++;
                        s.params.push_back(expr());
                    }
                }
                expect(")");
            }
            s.args = arglist();
            expect(";");
            std::vector<double> pv;
            for (auto &e : s.params) pv.push_back(eval(e, {}, line));
            // broadcast over whole registers
            size_t width = 1;
            for (const Arg &a : s.args)
                if (a.index < 0) {
                    const size_t w = qubits(a, line).size();
                    if (width != 1 && w != width) error("registers of different sizes", line);
                    width = w;
                }
            for (size_t k = 0; k < width; k++) {
                std::vector<int> qs;
                for (const Arg &a : s.args) {
                    const std::vector<int> all = qubits(a, line);
                    qs.push_back(a.index < 0 ? all[k] : all[0]);
                }
                apply(s.name, pv, qs, line);
            }
        }
    }

    double eval(const ExprP &e, const std::map<std::string, double> &env, int line) const {
        try {
            return e->eval(env);
        } catch (const ParseError &x) {
            error(x.what(), line);
        }
    }

    std::vector<int> qubits(const Arg &a, int line) const {
        auto it = qregs_.find(a.reg);
        if (it == qregs_.end()) error("unknown quantum register '" + a.reg + "'", line);
        if (a.index >= 0) {
            if (a.index >= it->second.second) error("index out of range for '" + a.reg + "'", line);
            return {it->second.first + (int)a.index};
        }
        std::vector<int> v;
        for (int k = 0; k < it->second.second; k++) v.push_back(it->second.first + k);
        return v;
    }

    void push(int op, int q0, int q1, double a, double b, double c) {
        qsim_gate g;
        std::memset(&g, 0, sizeof(g));
        g.op = (uint16_t)op;
        g.q0 = (uint32_t)q0;
        g.q1 = (uint32_t)q1;
        g.p[0] = a;
        g.p[1] = b;
        g.p[2] = c;
        gates.push_back(g);
    }
    void push_c1(int q, const double *m8) {  // 2x2 complex, row-major (re, im)
        qsim_gate g;
        std::memset(&g, 0, sizeof(g));
        g.op = QSIM_OP_C1;
        g.q0 = (uint32_t)q;
        g.mat = (uint32_t)mats.size();
        mats.insert(mats.end(), m8, m8 + 8);
        gates.push_back(g);
    }

    // X^t = ((1 + e^{i pi t}) I + (1 - e^{i pi t}) X) / 2 (principal power: t = 1
    // is X, t = 1/2 the sqrt(X) of `sx`), as a 2x2 complex matrix (re, im).
    static void xpow(double t, double *m8) {
        const double kPi = 3.14159265358979323846;
        // e^{i pi t}, exact where it has an exact value (X and sqrt(X) stay exact)
        double cr = std::cos(kPi * t), ci = std::sin(kPi * t);
        if (t == 1.0) cr = -1.0, ci = 0.0;
        if (t == 0.5 || t == -0.5) cr = 0.0, ci = t > 0 ? 1.0 : -1.0;
        const double d[2] = {(1 + cr) / 2, ci / 2}, o[2] = {(1 - cr) / 2, -ci / 2};
        m8[0] = d[0]; m8[1] = d[1]; m8[2] = o[0]; m8[3] = o[1];
        m8[4] = o[0]; m8[5] = o[1]; m8[6] = d[0]; m8[7] = d[1];
    }
    // Controlled-U on (control c, target t) as a C2 record: |0><0| (x) I + |1><1| (x) U
    // in the local basis l = b_c + 2 b_t.
    void push_controlled(int c, int t, const double *u8) {
        double m[32] = {0};
        auto set = [&](int r, int col, double re, double im) {
            m[2 * (4 * r + col)] = re;
            m[2 * (4 * r + col) + 1] = im;
        };
        set(0, 0, 1, 0);
        set(2, 2, 1, 0);
        for (int i = 0; i < 2; i++)      // target bit (row) with the control bit 1
            for (int j = 0; j < 2; j++)  // target bit (column)
                set(1 + 2 * i, 1 + 2 * j, u8[2 * (2 * i + j)], u8[2 * (2 * i + j) + 1]);
        qsim_gate g;
        std::memset(&g, 0, sizeof(g));
        g.op = QSIM_OP_C2;
        g.q0 = (uint32_t)c;
        g.q1 = (uint32_t)t;
        g.mat = (uint32_t)mats.size();
        mats.insert(mats.end(), m, m + 32);
        gates.push_back(g);
    }
    // X^t on `target` controlled by every qubit of `ctl`, exactly (no relative
    // phase), by the recursion of Barenco et al., Phys. Rev. A 52, 3457 (1995),
    // Lemma 7.5: with V = X^{t/2} and c the last control,
    //   C^k(X^t) = C^{k-1}(V) . C^{k-1}(X)[-> c] . C_c(V^dagger) . C^{k-1}(X)[-> c] . C_c(V)
    // (rightmost first): the two inner gates flip c only when the other controls
    // are all 1, so the target receives V V = X^t exactly when every control is 1
    // and V V^dagger = I or nothing otherwise.
    void multi_controlled_xpow(const std::vector<int> &ctl, int target, double t) {
        double u[8];
        if (ctl.size() == 1) {
            xpow(t, u);
            push_controlled(ctl[0], target, u);
            return;
        }
        const int c = ctl.back();
        const std::vector<int> rest(ctl.begin(), ctl.end() - 1);
        xpow(t / 2, u);
        push_controlled(c, target, u);
        multi_controlled_xpow(rest, c, 1.0);
        xpow(-t / 2, u);
        push_controlled(c, target, u);
        multi_controlled_xpow(rest, c, 1.0);
        multi_controlled_xpow(rest, target, t / 2);
    }

    // One gate on resolved qubits: a built-in of qelib1, or a user definition.
    void apply(const std::string &name, const std::vector<double> &p, const std::vector<int> &q, int line) {
        struct B {
            int op, nq, np;
        };
        static const std::map<std::string, B> builtin = {
            {"id", {QSIM_OP_ID, 1, 0}},      {"x", {QSIM_OP_X, 1, 0}},        {"y", {QSIM_OP_Y, 1, 0}},
            {"z", {QSIM_OP_Z, 1, 0}},        {"h", {QSIM_OP_H, 1, 0}},        {"s", {QSIM_OP_S, 1, 0}},
            {"sdg", {QSIM_OP_SDG, 1, 0}},    {"t", {QSIM_OP_T, 1, 0}},        {"tdg", {QSIM_OP_TDG, 1, 0}},
            {"rx", {QSIM_OP_RX, 1, 1}},      {"ry", {QSIM_OP_RY, 1, 1}},      {"rz", {QSIM_OP_RZ, 1, 1}},
            {"u1", {QSIM_OP_U1, 1, 1}},      {"p", {QSIM_OP_U1, 1, 1}},       {"u2", {QSIM_OP_U2, 1, 2}},
            {"u3", {QSIM_OP_U3, 1, 3}},      {"u", {QSIM_OP_U3, 1, 3}},       {"U", {QSIM_OP_U3, 1, 3}},
            {"cx", {QSIM_OP_CX, 2, 0}},      {"CX", {QSIM_OP_CX, 2, 0}},      {"cy", {QSIM_OP_CY, 2, 0}},
            {"cz", {QSIM_OP_CZ, 2, 0}},      {"ch", {QSIM_OP_CH, 2, 0}},      {"swap", {QSIM_OP_SWAP, 2, 0}},
            {"crx", {QSIM_OP_CRX, 2, 1}},    {"cry", {QSIM_OP_CRY, 2, 1}},    {"crz", {QSIM_OP_CRZ, 2, 1}},
            {"cu1", {QSIM_OP_CU1, 2, 1}},    {"cp", {QSIM_OP_CU1, 2, 1}},     {"cu3", {QSIM_OP_CU3, 2, 3}},
            {"rxx", {QSIM_OP_RXX, 2, 1}},    {"rzz", {QSIM_OP_RZZ, 2, 1}},
        };
        auto check = [&](size_t nq, size_t np) {
            if (q.size() != nq) error("'" + name + "' takes " + std::to_string(nq) + " qubit(s)", line);
            if (p.size() != np) error("'" + name + "' takes " + std::to_string(np) + " parameter(s)", line);
            for (size_t a = 0; a < q.size(); a++)
                for (size_t b = a + 1; b < q.size(); b++)
                    if (q[a] == q[b]) error("'" + name + "' on a repeated qubit", line);
        };
        auto it = builtin.find(name);
        if (it != builtin.end()) {
            check(it->second.nq, it->second.np);
            push(it->second.op, q[0], q.size() > 1 ? q[1] : 0, p.size() > 0 ? p[0] : 0, p.size() > 1 ? p[1] : 0,
                 p.size() > 2 ? p[2] : 0);
            return;
        }
        if (name == "sx" || name == "sxdg") {  // sqrt(X) = ((1+i) I + (1-i) X) / 2, and its adjoint
            check(1, 0);
            const double s = name == "sx" ? 1.0 : -1.0;
            const double m[8] = {0.5, 0.5 * s, 0.5, -0.5 * s, 0.5, -0.5 * s, 0.5, 0.5 * s};
            push_c1(q[0], m);
            return;
        }
        if (name == "ccx") {  // Toffoli as 1- and 2-qubit gates (exact, phase included)
            check(3, 0);
            const int a = q[0], b = q[1], c = q[2];
            push(QSIM_OP_H, c, 0, 0, 0, 0);
            push(QSIM_OP_CX, b, c, 0, 0, 0);
            push(QSIM_OP_TDG, c, 0, 0, 0, 0);
            push(QSIM_OP_CX, a, c, 0, 0, 0);
            push(QSIM_OP_T, c, 0, 0, 0, 0);
            push(QSIM_OP_CX, b, c, 0, 0, 0);
            push(QSIM_OP_TDG, c, 0, 0, 0, 0);
            push(QSIM_OP_CX, a, c, 0, 0, 0);
            push(QSIM_OP_T, b, 0, 0, 0, 0);
            push(QSIM_OP_T, c, 0, 0, 0, 0);
            push(QSIM_OP_H, c, 0, 0, 0, 0);
            push(QSIM_OP_CX, a, b, 0, 0, 0);
            push(QSIM_OP_T, a, 0, 0, 0, 0);
            push(QSIM_OP_TDG, b, 0, 0, 0, 0);
            push(QSIM_OP_CX, a, b, 0, 0, 0);
            return;
        }
        if (name == "cswap") {  // Fredkin: CX(c,b) Toffoli(a,b,c) CX(c,b)
            check(3, 0);
            push(QSIM_OP_CX, q[2], q[1], 0, 0, 0);
            apply("ccx", {}, {q[0], q[1], q[2]}, line);
            push(QSIM_OP_CX, q[2], q[1], 0, 0, 0);
            return;
        }
        if (name == "c3x" || name == "c4x" || name == "c3sqrtx") {
            // exact multi-controlled X^t (t = 1, or 1/2 for sqrt(X)), phase included
            const size_t nc = name == "c4x" ? 4 : 3;
            check(nc + 1, 0);
            const std::vector<int> ctl(q.begin(), q.begin() + nc);
            multi_controlled_xpow(ctl, q[nc], name == "c3sqrtx" ? 0.5 : 1.0);
            return;
        }
        if (name == "rccx") {
            // relative-phase Toffoli (Margolus form in Clifford+T; Maslov, Phys. Rev. A
            // 93, 022311 (2016)): Toffoli followed by the phases -i on |a b c> = |110>,
            // +i on |111> and -1 on |101> (a, b controls, c target)
            check(3, 0);
            const int a = q[0], b = q[1], c = q[2];
            push(QSIM_OP_H, c, 0, 0, 0, 0);
            push(QSIM_OP_T, c, 0, 0, 0, 0);
            push(QSIM_OP_CX, b, c, 0, 0, 0);
            push(QSIM_OP_TDG, c, 0, 0, 0, 0);
            push(QSIM_OP_CX, a, c, 0, 0, 0);
            push(QSIM_OP_T, c, 0, 0, 0, 0);
            push(QSIM_OP_CX, b, c, 0, 0, 0);
            push(QSIM_OP_TDG, c, 0, 0, 0, 0);
            push(QSIM_OP_H, c, 0, 0, 0, 0);
            return;
        }
        if (name == "rc3x") {
            // relative-phase 3-controlled X (Maslov 2016, Clifford+T): C3X followed by
            // the phases +i on |a b c d> = |1100>, -i on |1101> and -1 on |1111>
            // (a, b, c controls, d target)
            check(4, 0);
            const int a = q[0], b = q[1], c = q[2], d = q[3];
            push(QSIM_OP_H, d, 0, 0, 0, 0);
            push(QSIM_OP_T, d, 0, 0, 0, 0);
            push(QSIM_OP_CX, c, d, 0, 0, 0);
            push(QSIM_OP_TDG, d, 0, 0, 0, 0);
            push(QSIM_OP_H, d, 0, 0, 0, 0);
            push(QSIM_OP_CX, a, d, 0, 0, 0);
            push(QSIM_OP_T, d, 0, 0, 0, 0);
            push(QSIM_OP_CX, b, d, 0, 0, 0);
            push(QSIM_OP_TDG, d, 0, 0, 0, 0);
            push(QSIM_OP_CX, a, d, 0, 0, 0);
            push(QSIM_OP_T, d, 0, 0, 0, 0);
            push(QSIM_OP_CX, b, d, 0, 0, 0);
            push(QSIM_OP_TDG, d, 0, 0, 0, 0);
            push(QSIM_OP_H, d, 0, 0, 0, 0);
            push(QSIM_OP_T, d, 0, 0, 0, 0);
            push(QSIM_OP_CX, c, d, 0, 0, 0);
            push(QSIM_OP_TDG, d, 0, 0, 0, 0);
            push(QSIM_OP_H, d, 0, 0, 0, 0);
            return;
        }
        auto d = defs_.find(name);
        if (d == defs_.end()) error("unknown gate '" + name + "'", line);
        const GateDef &g = d->second;
        check(g.qargs.size(), g.params.size());
        if (++depth_ > 64) error("gate definitions nested too deep", line);
        std::map<std::string, double> env;
        for (size_t k = 0; k < g.params.size(); k++) env[g.params[k]] = p[k];
        std::map<std::string, int> qmap;
        for (size_t k = 0; k < g.qargs.size(); k++) qmap[g.qargs[k]] = q[k];
        for (const Stmt &s : g.body) {
            std::vector<double> pv;
            for (auto &e : s.params) pv.push_back(eval(e, env, s.line));
            std::vector<int> qs;
            for (const Arg &a : s.args) {
                auto it2 = qmap.find(a.reg);
                if (it2 == qmap.end() || a.index >= 0) error("bad argument '" + a.reg + "' in gate body", s.line);
                qs.push_back(it2->second);
            }
            apply(s.name, pv, qs, s.line);
        }
        depth_--;
    }
};

}  // namespace

extern "C" qsim_status qsim_parse_qasm(const char *text, size_t len, qsim_gate *gates, size_t cap_gates,
                                       size_t *n_gates, double *mats, size_t cap_mats, size_t *n_mats,
                                       int *n_qubits, char *err, size_t err_cap) {
    auto set_err = [&](const std::string &m) {
        if (err && err_cap) {
            const size_t k = std::min(err_cap - 1, m.size());
            std::memcpy(err, m.data(), k);
            err[k] = 0;
        }
    };
    set_err("");
    if (!text && len) {
        set_err("null text");
        return QSIM_E_INVAL;
    }
    try {
        Parser p(text ? text : "", len);
        p.run();
        if (n_gates) *n_gates = p.gates.size();
        if (n_mats) *n_mats = p.mats.size();
        if (n_qubits) *n_qubits = p.n_qubits;
        if (p.gates.size() > cap_gates || p.mats.size() > cap_mats) {
            set_err("output capacity too small");
            return QSIM_E_INVAL;
        }
        if (!p.gates.empty()) std::memcpy(gates, p.gates.data(), p.gates.size() * sizeof(qsim_gate));
        if (!p.mats.empty()) std::memcpy(mats, p.mats.data(), p.mats.size() * sizeof(double));
        return QSIM_OK;
    } catch (const ParseError &e) {
        set_err(e.what());
        return QSIM_E_INVAL;
    } catch (const std::bad_alloc &) {
        set_err("out of host memory");
        return QSIM_E_OOM;
    }
}
