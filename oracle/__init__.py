"""CPU oracle for exact big-integer multiplication (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import, call, link or execute anything in this
package.  The library's product path never touches it, and this package never
imports the library.

Contents, each pinned by the ``-m "not gpu"`` tests:

* ``schoolbook.c`` / ``native`` - the plain definition of the product w = u v
  (Section 1) as a limb-by-limb schoolbook with a 64-bit accumulator.
* ``toom`` - a plain recursive B-way Toom-Cook on Python integers that takes
  the paper's steps in order (split, evaluation at 0 and +-2^j via even and
  odd parts, pointwise products, even-odd combine, Newton divided
  differences, Newton-to-monomial conversion, recomposition) and exposes every
  intermediate.
* ``vandermonde`` - exact rational inversion of the Vandermonde matrix, the
  alternative route to the coefficients named at the end of Section 3.
* ``residues`` - products checked modulo three 61-bit primes.

No function here is "parity unpinned": each one is checked against brute
force, closed forms, a library routine or an independent route.
"""
