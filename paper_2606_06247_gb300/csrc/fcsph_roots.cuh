// Generated by gen_roots.py: cos and sin of 2 pi e / N for the composite
// register-DFT sizes N.  Do not edit by hand.
#pragma once

namespace fcsph {

template <int N> __device__ __forceinline__ double rcos(int e);
template <int N> __device__ __forceinline__ double rsin(int e);

template <> __device__ __forceinline__ double rcos<10>(int e) {
  switch (((e % 10) + 10) % 10) {
    case 0: return 1.0;
    case 1: return 0.80901699437494742;
    case 2: return 0.30901699437494742;
    case 3: return -0.30901699437494742;
    case 4: return -0.80901699437494742;
    case 5: return -1.0;
    case 6: return -0.80901699437494742;
    case 7: return -0.30901699437494742;
    case 8: return 0.30901699437494742;
    case 9: return 0.80901699437494742;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double rsin<10>(int e) {
  switch (((e % 10) + 10) % 10) {
    case 0: return 0.0;
    case 1: return 0.58778525229247313;
    case 2: return 0.95105651629515357;
    case 3: return 0.95105651629515357;
    case 4: return 0.58778525229247313;
    case 5: return 4.1340642196527976e-43;
    case 6: return -0.58778525229247313;
    case 7: return -0.95105651629515357;
    case 8: return -0.95105651629515357;
    case 9: return -0.58778525229247313;
    default: return 0.0;
  }
}

template <> __device__ __forceinline__ double rcos<14>(int e) {
  switch (((e % 14) + 14) % 14) {
    case 0: return 1.0;
    case 1: return 0.90096886790241913;
    case 2: return 0.62348980185873353;
    case 3: return 0.2225209339563144;
    case 4: return -0.2225209339563144;
    case 5: return -0.62348980185873353;
    case 6: return -0.90096886790241913;
    case 7: return -1.0;
    case 8: return -0.90096886790241913;
    case 9: return -0.62348980185873353;
    case 10: return -0.2225209339563144;
    case 11: return 0.2225209339563144;
    case 12: return 0.62348980185873353;
    case 13: return 0.90096886790241913;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double rsin<14>(int e) {
  switch (((e % 14) + 14) % 14) {
    case 0: return 0.0;
    case 1: return 0.43388373911755812;
    case 2: return 0.78183148246802981;
    case 3: return 0.97492791218182361;
    case 4: return 0.97492791218182361;
    case 5: return 0.78183148246802981;
    case 6: return 0.43388373911755812;
    case 7: return 4.1340642196527976e-43;
    case 8: return -0.43388373911755812;
    case 9: return -0.78183148246802981;
    case 10: return -0.97492791218182361;
    case 11: return -0.97492791218182361;
    case 12: return -0.78183148246802981;
    case 13: return -0.43388373911755812;
    default: return 0.0;
  }
}

template <> __device__ __forceinline__ double rcos<15>(int e) {
  switch (((e % 15) + 15) % 15) {
    case 0: return 1.0;
    case 1: return 0.9135454576426009;
    case 2: return 0.66913060635885821;
    case 3: return 0.30901699437494742;
    case 4: return -0.10452846326765347;
    case 5: return -0.5;
    case 6: return -0.80901699437494742;
    case 7: return -0.97814760073380564;
    case 8: return -0.97814760073380564;
    case 9: return -0.80901699437494742;
    case 10: return -0.5;
    case 11: return -0.10452846326765347;
    case 12: return 0.30901699437494742;
    case 13: return 0.66913060635885821;
    case 14: return 0.9135454576426009;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double rsin<15>(int e) {
  switch (((e % 15) + 15) % 15) {
    case 0: return 0.0;
    case 1: return 0.40673664307580021;
    case 2: return 0.74314482547739424;
    case 3: return 0.95105651629515357;
    case 4: return 0.99452189536827334;
    case 5: return 0.86602540378443865;
    case 6: return 0.58778525229247313;
    case 7: return 0.20791169081775934;
    case 8: return -0.20791169081775934;
    case 9: return -0.58778525229247313;
    case 10: return -0.86602540378443865;
    case 11: return -0.99452189536827334;
    case 12: return -0.95105651629515357;
    case 13: return -0.74314482547739424;
    case 14: return -0.40673664307580021;
    default: return 0.0;
  }
}

template <> __device__ __forceinline__ double rcos<20>(int e) {
  switch (((e % 20) + 20) % 20) {
    case 0: return 1.0;
    case 1: return 0.95105651629515357;
    case 2: return 0.80901699437494742;
    case 3: return 0.58778525229247313;
    case 4: return 0.30901699437494742;
    case 5: return 2.0670321098263988e-43;
    case 6: return -0.30901699437494742;
    case 7: return -0.58778525229247313;
    case 8: return -0.80901699437494742;
    case 9: return -0.95105651629515357;
    case 10: return -1.0;
    case 11: return -0.95105651629515357;
    case 12: return -0.80901699437494742;
    case 13: return -0.58778525229247313;
    case 14: return -0.30901699437494742;
    case 15: return -6.9496731751441328e-41;
    case 16: return 0.30901699437494742;
    case 17: return 0.58778525229247313;
    case 18: return 0.80901699437494742;
    case 19: return 0.95105651629515357;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double rsin<20>(int e) {
  switch (((e % 20) + 20) % 20) {
    case 0: return 0.0;
    case 1: return 0.30901699437494742;
    case 2: return 0.58778525229247313;
    case 3: return 0.80901699437494742;
    case 4: return 0.95105651629515357;
    case 5: return 1.0;
    case 6: return 0.95105651629515357;
    case 7: return 0.80901699437494742;
    case 8: return 0.58778525229247313;
    case 9: return 0.30901699437494742;
    case 10: return 4.1340642196527976e-43;
    case 11: return -0.30901699437494742;
    case 12: return -0.58778525229247313;
    case 13: return -0.80901699437494742;
    case 14: return -0.95105651629515357;
    case 15: return -1.0;
    case 16: return -0.95105651629515357;
    case 17: return -0.80901699437494742;
    case 18: return -0.58778525229247313;
    case 19: return -0.30901699437494742;
    default: return 0.0;
  }
}

template <> __device__ __forceinline__ double rcos<21>(int e) {
  switch (((e % 21) + 21) % 21) {
    case 0: return 1.0;
    case 1: return 0.95557280578614073;
    case 2: return 0.82623877431599487;
    case 3: return 0.62348980185873353;
    case 4: return 0.36534102436639501;
    case 5: return 7.4730093586424254e-2;
    case 6: return -0.2225209339563144;
    case 7: return -0.5;
    case 8: return -0.73305187182982633;
    case 9: return -0.90096886790241913;
    case 10: return -0.98883082622512855;
    case 11: return -0.98883082622512855;
    case 12: return -0.90096886790241913;
    case 13: return -0.73305187182982633;
    case 14: return -0.5;
    case 15: return -0.2225209339563144;
    case 16: return 7.4730093586424254e-2;
    case 17: return 0.36534102436639501;
    case 18: return 0.62348980185873353;
    case 19: return 0.82623877431599487;
    case 20: return 0.95557280578614073;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double rsin<21>(int e) {
  switch (((e % 21) + 21) % 21) {
    case 0: return 0.0;
    case 1: return 0.29475517441090422;
    case 2: return 0.56332005806362203;
    case 3: return 0.78183148246802981;
    case 4: return 0.93087374864420426;
    case 5: return 0.99720379718118015;
    case 6: return 0.97492791218182361;
    case 7: return 0.86602540378443865;
    case 8: return 0.68017273777091939;
    case 9: return 0.43388373911755812;
    case 10: return 0.14904226617617445;
    case 11: return -0.14904226617617445;
    case 12: return -0.43388373911755812;
    case 13: return -0.68017273777091939;
    case 14: return -0.86602540378443865;
    case 15: return -0.97492791218182361;
    case 16: return -0.99720379718118015;
    case 17: return -0.93087374864420426;
    case 18: return -0.78183148246802981;
    case 19: return -0.56332005806362203;
    case 20: return -0.29475517441090422;
    default: return 0.0;
  }
}

template <> __device__ __forceinline__ double rcos<25>(int e) {
  switch (((e % 25) + 25) % 25) {
    case 0: return 1.0;
    case 1: return 0.96858316112863112;
    case 2: return 0.87630668004386359;
    case 3: return 0.72896862742141152;
    case 4: return 0.53582679497899662;
    case 5: return 0.30901699437494742;
    case 6: return 6.2790519529313376e-2;
    case 7: return -0.18738131458572463;
    case 8: return -0.42577929156507265;
    case 9: return -0.63742398974868971;
    case 10: return -0.80901699437494742;
    case 11: return -0.9297764858882514;
    case 12: return -0.99211470131447783;
    case 13: return -0.99211470131447783;
    case 14: return -0.9297764858882514;
    case 15: return -0.80901699437494742;
    case 16: return -0.63742398974868971;
    case 17: return -0.42577929156507265;
    case 18: return -0.18738131458572463;
    case 19: return 6.2790519529313376e-2;
    case 20: return 0.30901699437494742;
    case 21: return 0.53582679497899662;
    case 22: return 0.72896862742141152;
    case 23: return 0.87630668004386359;
    case 24: return 0.96858316112863112;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double rsin<25>(int e) {
  switch (((e % 25) + 25) % 25) {
    case 0: return 0.0;
    case 1: return 0.24868988716485479;
    case 2: return 0.48175367410171527;
    case 3: return 0.68454710592868867;
    case 4: return 0.84432792550201508;
    case 5: return 0.95105651629515357;
    case 6: return 0.99802672842827156;
    case 7: return 0.98228725072868868;
    case 8: return 0.90482705246601953;
    case 9: return 0.77051324277578923;
    case 10: return 0.58778525229247313;
    case 11: return 0.36812455268467796;
    case 12: return 0.12533323356430425;
    case 13: return -0.12533323356430425;
    case 14: return -0.36812455268467796;
    case 15: return -0.58778525229247313;
    case 16: return -0.77051324277578923;
    case 17: return -0.90482705246601953;
    case 18: return -0.98228725072868868;
    case 19: return -0.99802672842827156;
    case 20: return -0.95105651629515357;
    case 21: return -0.84432792550201508;
    case 22: return -0.68454710592868867;
    case 23: return -0.48175367410171527;
    case 24: return -0.24868988716485479;
    default: return 0.0;
  }
}

template <> __device__ __forceinline__ double rcos<27>(int e) {
  switch (((e % 27) + 27) % 27) {
    case 0: return 1.0;
    case 1: return 0.97304487057982384;
    case 2: return 0.89363264032341225;
    case 3: return 0.76604444311897804;
    case 4: return 0.59715859170278616;
    case 5: return 0.39607976603915682;
    case 6: return 0.17364817766693035;
    case 7: return -5.8144828910475829e-2;
    case 8: return -0.28680323271109025;
    case 9: return -0.5;
    case 10: return -0.68624163786873359;
    case 11: return -0.83548781141293642;
    case 12: return -0.93969262078590838;
    case 13: return -0.99323835774194299;
    case 14: return -0.99323835774194299;
    case 15: return -0.93969262078590838;
    case 16: return -0.83548781141293642;
    case 17: return -0.68624163786873359;
    case 18: return -0.5;
    case 19: return -0.28680323271109025;
    case 20: return -5.8144828910475829e-2;
    case 21: return 0.17364817766693035;
    case 22: return 0.39607976603915682;
    case 23: return 0.59715859170278616;
    case 24: return 0.76604444311897804;
    case 25: return 0.89363264032341225;
    case 26: return 0.97304487057982384;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double rsin<27>(int e) {
  switch (((e % 27) + 27) % 27) {
    case 0: return 0.0;
    case 1: return 0.23061587074244018;
    case 2: return 0.44879918020046217;
    case 3: return 0.64278760968653933;
    case 4: return 0.80212319275504379;
    case 5: return 0.91821610688027401;
    case 6: return 0.98480775301220806;
    case 7: return 0.99830815827126821;
    case 8: return 0.95798951231548887;
    case 9: return 0.86602540378443865;
    case 10: return 0.7273736415730487;
    case 11: return 0.54950897807080604;
    case 12: return 0.34202014332566873;
    case 13: return 0.11609291412523023;
    case 14: return -0.11609291412523023;
    case 15: return -0.34202014332566873;
    case 16: return -0.54950897807080604;
    case 17: return -0.7273736415730487;
    case 18: return -0.86602540378443865;
    case 19: return -0.95798951231548887;
    case 20: return -0.99830815827126821;
    case 21: return -0.98480775301220806;
    case 22: return -0.91821610688027401;
    case 23: return -0.80212319275504379;
    case 24: return -0.64278760968653933;
    case 25: return -0.44879918020046217;
    case 26: return -0.23061587074244018;
    default: return 0.0;
  }
}

template <> __device__ __forceinline__ double rcos<28>(int e) {
  switch (((e % 28) + 28) % 28) {
    case 0: return 1.0;
    case 1: return 0.97492791218182361;
    case 2: return 0.90096886790241913;
    case 3: return 0.78183148246802981;
    case 4: return 0.62348980185873353;
    case 5: return 0.43388373911755812;
    case 6: return 0.2225209339563144;
    case 7: return 2.0670321098263988e-43;
    case 8: return -0.2225209339563144;
    case 9: return -0.43388373911755812;
    case 10: return -0.62348980185873353;
    case 11: return -0.78183148246802981;
    case 12: return -0.90096886790241913;
    case 13: return -0.97492791218182361;
    case 14: return -1.0;
    case 15: return -0.97492791218182361;
    case 16: return -0.90096886790241913;
    case 17: return -0.78183148246802981;
    case 18: return -0.62348980185873353;
    case 19: return -0.43388373911755812;
    case 20: return -0.2225209339563144;
    case 21: return 2.2338764406549883e-41;
    case 22: return 0.2225209339563144;
    case 23: return 0.43388373911755812;
    case 24: return 0.62348980185873353;
    case 25: return 0.78183148246802981;
    case 26: return 0.90096886790241913;
    case 27: return 0.97492791218182361;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double rsin<28>(int e) {
  switch (((e % 28) + 28) % 28) {
    case 0: return 0.0;
    case 1: return 0.2225209339563144;
    case 2: return 0.43388373911755812;
    case 3: return 0.62348980185873353;
    case 4: return 0.78183148246802981;
    case 5: return 0.90096886790241913;
    case 6: return 0.97492791218182361;
    case 7: return 1.0;
    case 8: return 0.97492791218182361;
    case 9: return 0.90096886790241913;
    case 10: return 0.78183148246802981;
    case 11: return 0.62348980185873353;
    case 12: return 0.43388373911755812;
    case 13: return 0.2225209339563144;
    case 14: return 4.1340642196527976e-43;
    case 15: return -0.2225209339563144;
    case 16: return -0.43388373911755812;
    case 17: return -0.62348980185873353;
    case 18: return -0.78183148246802981;
    case 19: return -0.90096886790241913;
    case 20: return -0.97492791218182361;
    case 21: return -1.0;
    case 22: return -0.97492791218182361;
    case 23: return -0.90096886790241913;
    case 24: return -0.78183148246802981;
    case 25: return -0.62348980185873353;
    case 26: return -0.43388373911755812;
    case 27: return -0.2225209339563144;
    default: return 0.0;
  }
}

template <> __device__ __forceinline__ double rcos<30>(int e) {
  switch (((e % 30) + 30) % 30) {
    case 0: return 1.0;
    case 1: return 0.97814760073380564;
    case 2: return 0.9135454576426009;
    case 3: return 0.80901699437494742;
    case 4: return 0.66913060635885821;
    case 5: return 0.5;
    case 6: return 0.30901699437494742;
    case 7: return 0.10452846326765347;
    case 8: return -0.10452846326765347;
    case 9: return -0.30901699437494742;
    case 10: return -0.5;
    case 11: return -0.66913060635885821;
    case 12: return -0.80901699437494742;
    case 13: return -0.9135454576426009;
    case 14: return -0.97814760073380564;
    case 15: return -1.0;
    case 16: return -0.97814760073380564;
    case 17: return -0.9135454576426009;
    case 18: return -0.80901699437494742;
    case 19: return -0.66913060635885821;
    case 20: return -0.5;
    case 21: return -0.30901699437494742;
    case 22: return -0.10452846326765347;
    case 23: return 0.10452846326765347;
    case 24: return 0.30901699437494742;
    case 25: return 0.5;
    case 26: return 0.66913060635885821;
    case 27: return 0.80901699437494742;
    case 28: return 0.9135454576426009;
    case 29: return 0.97814760073380564;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double rsin<30>(int e) {
  switch (((e % 30) + 30) % 30) {
    case 0: return 0.0;
    case 1: return 0.20791169081775934;
    case 2: return 0.40673664307580021;
    case 3: return 0.58778525229247313;
    case 4: return 0.74314482547739424;
    case 5: return 0.86602540378443865;
    case 6: return 0.95105651629515357;
    case 7: return 0.99452189536827334;
    case 8: return 0.99452189536827334;
    case 9: return 0.95105651629515357;
    case 10: return 0.86602540378443865;
    case 11: return 0.74314482547739424;
    case 12: return 0.58778525229247313;
    case 13: return 0.40673664307580021;
    case 14: return 0.20791169081775934;
    case 15: return 4.1340642196527976e-43;
    case 16: return -0.20791169081775934;
    case 17: return -0.40673664307580021;
    case 18: return -0.58778525229247313;
    case 19: return -0.74314482547739424;
    case 20: return -0.86602540378443865;
    case 21: return -0.95105651629515357;
    case 22: return -0.99452189536827334;
    case 23: return -0.99452189536827334;
    case 24: return -0.95105651629515357;
    case 25: return -0.86602540378443865;
    case 26: return -0.74314482547739424;
    case 27: return -0.58778525229247313;
    case 28: return -0.40673664307580021;
    case 29: return -0.20791169081775934;
    default: return 0.0;
  }
}

template <> __device__ __forceinline__ double rcos<35>(int e) {
  switch (((e % 35) + 35) % 35) {
    case 0: return 1.0;
    case 1: return 0.98392958859862966;
    case 2: return 0.93623487063973721;
    case 3: return 0.85844879360186612;
    case 4: return 0.75307146600361093;
    case 5: return 0.62348980185873353;
    case 6: return 0.47386866247299867;
    case 7: return 0.30901699437494742;
    case 8: return 0.13423326581765548;
    case 9: return -4.4864830350514925e-2;
    case 10: return -0.2225209339563144;
    case 11: return -0.39302503165392362;
    case 12: return -0.55089698145210252;
    case 13: return -0.69106264898686468;
    case 14: return -0.80901699437494742;
    case 15: return -0.90096886790241913;
    case 16: return -0.96396286069585329;
    case 17: return -0.99597429399523903;
    case 18: return -0.99597429399523903;
    case 19: return -0.96396286069585329;
    case 20: return -0.90096886790241913;
    case 21: return -0.80901699437494742;
    case 22: return -0.69106264898686468;
    case 23: return -0.55089698145210252;
    case 24: return -0.39302503165392362;
    case 25: return -0.2225209339563144;
    case 26: return -4.4864830350514925e-2;
    case 27: return 0.13423326581765548;
    case 28: return 0.30901699437494742;
    case 29: return 0.47386866247299867;
    case 30: return 0.62348980185873353;
    case 31: return 0.75307146600361093;
    case 32: return 0.85844879360186612;
    case 33: return 0.93623487063973721;
    case 34: return 0.98392958859862966;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double rsin<35>(int e) {
  switch (((e % 35) + 35) % 35) {
    case 0: return 0.0;
    case 1: return 0.17855689479863665;
    case 2: return 0.3513748240813427;
    case 3: return 0.51289927740590614;
    case 4: return 0.65793872593971261;
    case 5: return 0.78183148246802981;
    case 6: return 0.880595531856738;
    case 7: return 0.95105651629515357;
    case 8: return 0.99094976176793476;
    case 9: return 0.99899306654131465;
    case 10: return 0.97492791218182361;
    case 11: return 0.91952777255145064;
    case 12: return 0.83457325372130265;
    case 13: return 0.72279486382739153;
    case 14: return 0.58778525229247313;
    case 15: return 0.43388373911755812;
    case 16: return 0.26603684556667511;
    case 17: return 8.96393089034335e-2;
    case 18: return -8.96393089034335e-2;
    case 19: return -0.26603684556667511;
    case 20: return -0.43388373911755812;
    case 21: return -0.58778525229247313;
    case 22: return -0.72279486382739153;
    case 23: return -0.83457325372130265;
    case 24: return -0.91952777255145064;
    case 25: return -0.97492791218182361;
    case 26: return -0.99899306654131465;
    case 27: return -0.99094976176793476;
    case 28: return -0.95105651629515357;
    case 29: return -0.880595531856738;
    case 30: return -0.78183148246802981;
    case 31: return -0.65793872593971261;
    case 32: return -0.51289927740590614;
    case 33: return -0.3513748240813427;
    case 34: return -0.17855689479863665;
    default: return 0.0;
  }
}

}  // namespace fcsph
