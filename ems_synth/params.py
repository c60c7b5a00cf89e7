"""Material and numerical settings: the analogue of the EMSpice 3 YAML file.

The paper reads its material constants and numerical settings from a YAML
parameter file (Sec. IV-A, Fig. "Overall algorithmic flow") but prints only
symbols for them (Sec. III-A, III-D).  The values below are the readings this
project takes; each side (the CPU oracle and the CUDA library) marshals this
dict into its own structure.  Nothing here computes any part of the method.

Units are SI throughout (m, s, Pa, K, A, V, Ohm).
"""

EV = 1.602176634e-19          # J per eV (exact, SI 2019)
YEAR = 3.15576e7              # Julian year in s; the paper's 5e7 s = 1.5844 y (Sec. V-D)


def default_params(**overrides):
    """Return the default parameter dict; keyword arguments override entries."""
    p = dict(
        # physical constants (Sec. III-D symbols)
        e_charge=1.602176634e-19,   # C
        k_B=1.380649e-23,           # J/K
        Omega=1.18e-29,             # m^3, Cu atomic volume
        rho_Cu=2.25e-8,             # Ohm m, temperature independent here
        B_modulus=1.0e11,           # Pa; B in kappa and the bulk modulus in V_v
        Z_star=5.0,                 # effective charge number (calibrated)
        D0=1.0e-8,                  # m^2/s diffusivity prefactor (calibrated)
        Ea=0.8 * EV,                # J, activation energy
        Q_star=0.09 * EV,           # J, heat of transport (atoms go hot -> cold)
        delta=1.0e-9,               # m, void interface thickness (Robin BC)
        rho_Ta=1.8e-6,              # Ohm m, barrier resistivity
        h_Ta=5.0e-9,                # m, barrier thickness
        sigma_T=0.0,                # Pa, residual stress (initial condition)
        sigma_crit=500.0e6,         # Pa, critical (nucleation) stress
        T0=378.0,                   # K, uniform temperature when no map is set
        # schedule (Sec. V: outer aging steps; inner BE steps are a reading)
        horizon=10.0 * YEAR,        # s
        n_outer=64,
        n_inner=256,
        ir_fail_frac=0.10,          # failure = max IR drop >= 10 % of Vdd
        Vdd=1.0,                    # V
        # Krylov (Sec. IV-E)
        krylov_q=10,
        krylov_eta=1.0,
    )
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = v
    return p
