"""Constants of the table-driven FP64 exponential in pab_exp.cuh (exp_tab).

Tang's method (P. T. P. Tang, "Table-driven implementation of the exponential
function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989) with 32 table
entries: x = (32 m + j) ln2/32 + r, |r| <= ln2/64, e^x = 2^m 2^(j/32) e^r.
Printed here, from 60-digit decimal arithmetic, each correctly rounded to double:
  32/ln2;
  ln2/32 split as L1 + L2, L1 with 36 significant bits (N L1 exact for |N| < 2^17);
  2^(j/32) for j = 0..31.

    python gen_exp_tab.py
"""
import math
from decimal import Decimal, getcontext

getcontext().prec = 60
ln2 = Decimal(2).ln()
L = ln2 / 32
m, e = math.frexp(float(L))
L1 = math.ldexp(math.floor(m * 2 ** 36 + 0.5) / 2 ** 36, e)
L2 = float(L - Decimal(L1))
print(f"kInvL = {float(32 / ln2).hex()}")
print(f"kL1   = {L1.hex()}")
print(f"kL2   = {L2.hex()}")
tab = [float(Decimal(2) ** (Decimal(j) / 32)) for j in range(32)]
for i in range(0, 32, 4):
    print("    " + ", ".join(t.hex() for t in tab[i:i + 4]) + ",")
