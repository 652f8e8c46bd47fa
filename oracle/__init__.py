"""FP64 CPU oracle for the MUSCL-Hancock step of the vibrationally excited gas
model (Khrapov & Khoperskov 2018).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product path.  It shares no code with
the CUDA library.

* ``orc``        -- ctypes binding of the plain C step (``orc_muscl.c``).
* ``dispersion`` -- the dispersion relation of eq. 8 (quartic in omega) and the
                    linear eigenmode it implies.
* ``riemann``    -- exact Riemann solver of the frozen limit (Euler equations
                    with a passive vibrational energy).
"""
