"""Writes strip_cases.inc: the strip spread's accumulate step as one jump table per J.

For a hit whose window starts at unit-relative column sd (-7 <= sd <= 15), tap j
(0 <= j < J) of the window lands on column sd + j, and only the columns inside the
unit [0, 16) are kept.  The kernel keeps the 16 columns of a lane (two coils each)
in registers, so each start column needs its own instruction sequence with
compile-time register operands; a warp-uniform brx.idx (index sd + 7) jumps to it.
Operands: %0..%63 the accumulators (column k: %4k..%4k+3 = real and imaginary parts
of the lane's two coils), %64 the case index, %65..%72 the column weights w[0..7],
%73..%76 the weighted coil values (real, imaginary of the first coil, then the
second).  Run from this directory: python gen_strip_cases.py
"""
import os

W = 16
SD_MIN, SD_MAX = -7, 15


def case_lines(J):
    out = []
    for sd in range(SD_MIN, SD_MAX + 1):
        ins = []
        for j in range(J):
            col = sd + j
            if 0 <= col < W:
                for q in range(4):
                    ins.append("fma.rn.f32 %%%d, %%%d, %%%d, %%%d;" % (4 * col + q, 65 + j, 73 + q, 4 * col + q))
        ins.append("bra.uni SE;")
        out.append('        "S%d: %s\\n\\t"' % (sd - SD_MIN, " ".join(ins)))
    return out


def main():
    n = SD_MAX - SD_MIN + 1
    labels = ", ".join("S%d" % i for i in range(n))
    text = ["// Generated by gen_strip_cases.py (same directory); do not edit by hand.",
            "// strip_add_J<J>(acc, sd, w, y): acc[4 (sd + j) + q] += w[j] * y[q] for the taps j < J",
            "// whose column sd + j lies in [0, 16), q < 4; sd in [-7, 15] (warp-uniform).",
            "#pragma once", "", "namespace nj {", "",
            "template <int J>",
            "__device__ __forceinline__ void strip_add_J(float (&a)[64], int sd, const float (&w)[8], const float (&y)[4]);",
            ""]
    outs = ", ".join('"+f"(a[%d])' % k for k in range(64))
    ins = ", ".join(['"r"(sd + 7)'] + ['"f"(w[%d])' % j for j in range(8)] + ['"f"(y[%d])' % q for q in range(4)])
    for J in range(4, 9):
        text.append("template <>")
        text.append("__device__ __forceinline__ void strip_add_J<%d>(float (&a)[64], int sd, const float (&w)[8], "
                    "const float (&y)[4]) {" % J)
        text.append('    asm volatile("{\\n\\t"')
        text.append('        "st: .branchtargets %s;\\n\\t"' % labels)
        text.append('        "brx.idx.uni %64, st;\\n\\t"')
        text.extend(case_lines(J))
        text.append('        "SE:\\n\\t}"')
        text.append("        : " + outs)
        text.append("        : " + ins + ");")
        text.append("}")
        text.append("")
    text.append("}  // namespace nj")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "strip_cases.inc")
    with open(path, "w") as f:
        f.write("\n".join(text) + "\n")


if __name__ == "__main__":
    main()
