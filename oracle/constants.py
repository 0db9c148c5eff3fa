"""Physical constants of the model.

Table 1 (Appendix A, thermodynamic parameters) and the microphysics
constants of Section 2.1 (COSMO warm-rain closure: source terms Eq. (2.4)
and the rain terminal velocity).  Values are typed from the paper as printed.
"""
import math

# Table 1
c_l = 4218.0        # J/(kg K)  specific heat of liquid water
c_pd = 1005.0       # J/(kg K)  dry air, constant pressure
c_pv = 1850.0       # J/(kg K)  water vapour, constant pressure
c_vd = 718.0        # J/(kg K)  dry air, constant volume
c_vv = 1390.0       # J/(kg K)  water vapour, constant volume
e_ref = 610.7       # Pa        saturation vapour pressure at T_ref
L_ref = 2.835e6     # J/kg      latent heat at T_ref
R_d = 287.05        # J/(kg K)
R_v = 461.51        # J/(kg K)
T_ref = 273.15      # K
p_ref = 1.0e5       # Pa
epsilon = 0.622     # R_d / R_v as printed (not used on the hot path)

# Section 2.1, Eq. (2.4): S_ev, S_au (q_au = 0), S_ac coefficients
S_EV_A = 3.86e-3
S_EV_B = 9.41e-5
S_EV_C = 9.1
S_AU = 1.0e-3
Q_AU = 0.0
S_AC = 1.72

# Section 2.1: rain terminal velocity v_r = (pi rho_w N0)^(-1/8) v0 Gamma(4.5)/6 rho_r^(1/8)
N0_R = 8.0e6        # 1/m^4
V0_R = 130.0        # m^(1/2)/s
GAMMA_4_5 = math.gamma(4.5)

# Gravity is not in Table 1; the paper is silent on its value.  Reading: 9.81.
G_DEFAULT = 9.81
